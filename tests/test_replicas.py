"""The multi-GPU path's host logic with world size 2 over gloo on the CPU.

Frequencies are independent systems (Section II-D), so ranks share no data:
each solves its own block of frequencies and only the timing bookkeeping
crosses ranks (which units a rank takes, the slowest rank's time, barriers).
"""
import multiprocessing as mp
import os
import socket
import time
from datetime import timedelta

import pytest

from paper_1702_03781_gb300 import replicas


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _init(rank, ws, port, timeout_s):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=ws,
                            timeout=timedelta(seconds=timeout_s))
    return dist


def _bookkeeping_rank(rank, ws, port, q):
    dist = _init(rank, ws, port, 60)
    try:
        mine = list(replicas.shard(64, ws, rank))
        every = [None] * ws
        dist.all_gather_object(every, mine)
        # rank r's step took 10 + r ms: the job's step is the slowest rank's
        slowest = replicas.max_over_ranks(10.0 + rank)
        replicas.barrier()
        q.put((rank, replicas.world(), every, slowest, replicas.ms_per_unit(slowest, ws)))
    finally:
        dist.destroy_process_group()


def _put_and_exit(q, item):
    q.put(item)
    q.close()
    q.join_thread()  # the item is in the pipe before the process ends
    os._exit(0)


def _leaving_rank(rank, ws, port, q):
    _init(rank, ws, port, 5)
    replicas.barrier()
    if rank == 1:
        # leaves between steps, with no collective in flight
        _put_and_exit(q, (rank, "left"))
    t0 = time.monotonic()
    try:
        replicas.max_over_ranks(1.0)
        _put_and_exit(q, (rank, "no error"))
    except Exception as e:  # gloo reports the lost peer or the timeout
        _put_and_exit(q, (rank, "error", type(e).__name__, time.monotonic() - t0))


def _run(target, ws=2, wait_s=120):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=target, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    out = [q.get(timeout=wait_s) for _ in range(ws)]
    for p in procs:
        p.join(timeout=wait_s)
        if p.is_alive():
            p.kill()
    return {o[0]: o for o in out}


def test_shard_covers_every_unit_once():
    for n in (0, 1, 5, 63, 64, 65, 1000):
        for ws in (1, 2, 3, 4, 8):
            blocks = [replicas.shard(n, ws, r) for r in range(ws)]
            flat = [u for b in blocks for u in b]
            assert flat == list(range(n))
            sizes = [len(b) for b in blocks]
            assert max(sizes) - min(sizes) <= 1


def test_shard_rejects_bad_ranks():
    with pytest.raises(ValueError):
        replicas.shard(8, 2, 2)
    with pytest.raises(ValueError):
        replicas.shard(8, 0, 0)
    with pytest.raises(ValueError):
        replicas.shard(-1, 2, 0)


def test_single_process_needs_no_group():
    assert replicas.world() == (1, 0)
    assert replicas.max_over_ranks(3.5) == 3.5
    replicas.barrier()
    assert replicas.ms_per_unit(26.0, 2) == 13.0


def test_two_gloo_ranks_share_the_units_and_take_the_slowest_time():
    out = _run(_bookkeeping_rank)
    for rank in (0, 1):
        _, world, every, slowest, per_unit = out[rank]
        assert world == (2, rank)
        assert every == [list(range(0, 32)), list(range(32, 64))]
        assert slowest == 11.0
        assert per_unit == 5.5


def test_a_rank_that_leaves_ends_the_next_collective_with_an_error():
    out = _run(_leaving_rank)
    assert out[1][1] == "left"
    assert out[0][1] == "error", out[0]
    assert out[0][3] < 60.0
