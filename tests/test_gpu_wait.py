"""Bounded device waits: a wait that nothing releases ends by itself, the host
reads HARP_E_TIMEOUT, and the context keeps working.

The wait under test is the one every mbarrier wait of the tensor-core kernels
uses (a clock budget of 2^30 SM cycles, about 0.5 s at 2 GHz). Nothing here
faults or hangs the GPU: the unreleased wait gives up within its budget.
"""
import time

import numpy as np
import pytest
import torch

import oracle
from paper_1702_03781_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def harp():
    from paper_1702_03781_gb300 import build
    build.build()
    from paper_1702_03781_gb300.harp import Harp
    h = Harp(0, max_N=256, max_nrhs=64)
    yield h
    h.close()


def test_released_wait_returns_ok(harp):
    from paper_1702_03781_gb300.harp import HARP_OK
    t0 = time.perf_counter()
    assert harp.wait_check(True) == HARP_OK
    assert time.perf_counter() - t0 < 0.2


def test_unreleased_wait_times_out_and_context_stays_usable(harp):
    from paper_1702_03781_gb300.harp import HARP_E_TIMEOUT, HARP_OK
    t0 = time.perf_counter()
    assert harp.wait_check(False) == HARP_E_TIMEOUT
    dt = time.perf_counter() - t0
    # the budget is 2^30 cycles: 0.52 s at 2070 MHz, longer at lower clocks
    assert 0.1 < dt < 20.0, dt
    # the status word was cleared: a released wait and a mixed solve succeed
    assert harp.wait_check(True) == HARP_OK
    p = synth.tiny()
    d = "cuda:0"
    pos, coef, sb = (torch.from_numpy(p.pos).to(d), torch.from_numpy(p.coef).to(d),
                     torch.from_numpy(p.self_blocks).to(d))
    Z = harp.fill(pos, p.freq_hz, coef, sb, prec="mixed")
    X, info = harp.solve(Z, None, nrhs=p.Na, prec="mixed", max_iter=10)
    Xo = oracle.solve(oracle.fill(p.pos, p.freq_hz, p.coef, p.self_blocks), p.V)
    Xg = X.detach().cpu().numpy()
    assert np.linalg.norm(Xg - Xo) / np.linalg.norm(Xo) <= 1e-10
