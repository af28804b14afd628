"""The tile-shape knobs change how the work is cut, not what is computed:
  * fill_chunk (source MBFs staged per fill CTA) leaves every entry's
    arithmetic alone, so the complex64 fill is bit-identical for every
    chunk;
  * panel_rows (rows per CTA of the cluster panel) and splitk_max (K splits
    of the tensor-core products) reorder FP32 sums, so the refined solution
    must meet the mixed solve's bar against the FP64 oracle: relative
    Frobenius error <= 1e-10, backward error <= sqrt(N) 2^-53.
Also: the batch's device time (CUDA events on every worker stream) is
positive and no larger than the host's wall clock around the call, and the
options refuse values outside their ranges."""
import math
import time

import numpy as np
import pytest
import torch

import oracle
from paper_1702_03781_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H():
    from paper_1702_03781_gb300 import build
    build.build()
    from paper_1702_03781_gb300 import harp
    return harp


def _dev(p):
    d = "cuda:0"
    return (torch.from_numpy(p.pos).to(d), torch.from_numpy(p.coef).to(d),
            torch.from_numpy(p.self_blocks).to(d))


def test_option_ranges(H):
    with H.Harp(0, max_N=256, max_nrhs=16) as h:
        assert h.knob("panel_rows") == 192 and h.knob("fill_chunk") == 0
        assert h.knob("splitk_max") == 8 and h.knob("inverses") == 2
        for name, bad in (("panel_rows", 16), ("panel_rows", 512), ("fill_chunk", -1),
                          ("splitk_max", 0), ("splitk_max", 9), ("inverses", 3),
                          ("inverses", -1), ("fill_clusters", -1), ("fill_clusters", 65)):
            with pytest.raises(H.HarpError):
                h.set_knob(name, bad)
        h.set_knob("splitk_max", 2)
        assert h.knob("splitk_max") == 2


def test_fill_chunk_bit_identical(H):
    p = synth.station()
    pos, coef, sb = _dev(p)
    with H.Harp(0, max_N=p.N, max_nrhs=p.Na) as h:
        ref = h.fill(pos, p.freq_hz, coef, sb, prec="mixed").clone()
        for c in (1, 2, 5, 12, 40):
            h.set_knob("fill_chunk", c)
            Z = h.fill(pos, p.freq_hz, coef, sb, prec="mixed")
            assert torch.equal(Z, ref), c
        h.sync()


@pytest.mark.parametrize("knobs", [{"panel_rows": 96}, {"panel_rows": 384}, {"inverses": 0},
                                   {"fill_clusters": 2}, {"fill_clusters": 7},
                                   {"splitk_max": 1}, {"splitk_max": 2, "panel_rows": 128,
                                                       "fill_chunk": 3}])
def test_solve_meets_bar_for_every_knob(H, knobs):
    p = synth.station()
    pos, coef, sb = _dev(p)
    with H.Harp(0, max_N=p.N, max_nrhs=p.Na) as h:
        for name, v in knobs.items():
            h.set_knob(name, v)
        Z = h.fill(pos, p.freq_hz, coef, sb, prec="mixed")
        X, info = h.solve(Z, None, nrhs=p.Na, prec="mixed")
    Zo = oracle.fill(p.pos, p.freq_hz, p.coef, p.self_blocks)
    Xo = oracle.solve(Zo, p.V)
    Xg = X.cpu().numpy()
    assert np.linalg.norm(Xg - Xo) / np.linalg.norm(Xo) <= 1e-10
    assert info["resid"] <= math.sqrt(p.N) * 2.0 ** -53


def test_batch_device_time(H):
    probs = synth.wideband(64)
    d = "cuda:0"
    items = [H.BatchItem(torch.from_numpy(probs[i].pos).to(d), probs[i].freq_hz,
                         torch.from_numpy(probs[i].coef).to(d),
                         torch.from_numpy(probs[i].self_blocks).to(d)) for i in (30, 10, 0, 5)]
    ctxs = [H.Harp(0, max_N=max(it.N for it in items), max_nrhs=256) for _ in range(2)]
    H.solve_batch(ctxs, items, prec="mixed")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    H.solve_batch(ctxs, items, prec="mixed")
    wall_ms = 1e3 * (time.perf_counter() - t0)
    dev_ms = ctxs[0].batch_device_ms()
    assert all(it.status == 0 for it in items)
    assert 0.0 < dev_ms <= wall_ms + 0.5
    for c in ctxs:
        c.close()
