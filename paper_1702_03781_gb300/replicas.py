"""Replicas across GPUs: one process per GPU, each filling and solving its own
frequencies (Section II-D: every frequency is an independent system), with no
collective on the data path.

The only cross-rank steps are host bookkeeping:
  * which of the independent units (frequencies) a rank solves;
  * the whole-job time, taken as the slowest rank's;
  * barriers around the timed region.
They run over torch.distributed with any backend (NCCL on GPUs, gloo on CPU).
"""
from __future__ import annotations

import torch
import torch.distributed as dist


def world() -> tuple[int, int]:
    """(world_size, rank); (1, 0) without an initialised process group."""
    if dist.is_available() and dist.is_initialized():
        return dist.get_world_size(), dist.get_rank()
    return 1, 0


def shard(n_units: int, world_size: int, rank: int) -> range:
    """The contiguous block of units [0, n_units) that `rank` solves. Blocks
    differ in size by at most one (the first n_units % world_size ranks take
    one more); together they cover every unit once."""
    if world_size < 1 or not 0 <= rank < world_size:
        raise ValueError(f"rank {rank} outside a world of {world_size}")
    if n_units < 0:
        raise ValueError("n_units < 0")
    q, r = divmod(n_units, world_size)
    start = rank * q + min(rank, r)
    return range(start, start + q + (1 if rank < r else 0))


def max_over_ranks(x: float, device=None) -> float:
    """The largest x over all ranks (x itself in a single process). `device`
    is where the reduction tensor lives: a CUDA device for NCCL, the CPU for
    gloo."""
    ws, _ = world()
    if ws == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier() -> None:
    """Host barrier across ranks (no-op in a single process)."""
    ws, _ = world()
    if ws > 1:
        dist.barrier()


def ms_per_unit(slowest_ms_per_step: float, units_per_step: int) -> float:
    """Whole-job time per unit: all ranks' units in one step, over the slowest
    rank's step time."""
    if units_per_step < 1:
        raise ValueError("units_per_step < 1")
    return slowest_ms_per_step / units_per_step
