"""GPU parity of the FP32 factorisation with tournament pivoting (the
communication-avoiding LU panel), through the C ABI against the FP64 CPU
oracle.

Tournament pivoting factors the same matrix with another row order, so the
refined solution must meet the same bar as with partial pivoting:
relative Frobenius error <= 1e-10 against the oracle's X, for the port
right-hand sides, general right-hand sides and the transposed solve. The
panels it applies to (up to 4096 rows, 16 CTAs of at most 256 rows) cover
every panel of the station; larger ones fall back to partial pivoting, which
the 5120-unknown wideband case exercises. The FP32 mode keeps the backward
error bound stated in test_gpu_edge.py.
"""
import math

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
    h = Harp(0, max_N=5120, max_nrhs=256)
    h.set_pivot("tournament")
    yield h
    h.close()


def _dev(p):
    d = "cuda:0"
    return (torch.from_numpy(p.pos).to(d), torch.from_numpy(p.coef).to(d),
            torch.from_numpy(p.self_blocks).to(d))


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_pivot_option_round_trip(harp):
    assert harp.pivot_rule() == "tournament"
    harp.set_pivot("partial")
    assert harp.pivot_rule() == "partial"
    harp.set_pivot("tournament")
    with pytest.raises(KeyError):
        harp.set_pivot("rook")


@pytest.mark.parametrize("mk", [lambda: synth.tiny(), lambda: synth.small(37, 5, P=3, Q=2),
                                lambda: synth.small(70, 3, P=2, Q=4, seed_cfg=21),
                                lambda: synth.small(150, 9, P=3, Q=3, seed_cfg=61),
                                lambda: synth.station()])
def test_tournament_mixed_solve_matches_oracle(harp, mk):
    p = mk()
    pos, coef, sb = _dev(p)
    Z = harp.fill(pos, p.freq_hz, coef, sb, prec="mixed")
    X, info = harp.solve(Z, None, nrhs=p.Na, prec="mixed", max_iter=10)
    Zo = oracle.fill(p.pos, p.freq_hz, p.coef, p.self_blocks)
    assert _rel(X.cpu().numpy(), oracle.solve(Zo, p.V)) <= 1e-10
    assert info["resid"] <= math.sqrt(p.N) * 2.0 ** -53


def test_tournament_general_rhs_and_transpose(harp):
    p = synth.small(110, 7, P=2, Q=2, seed_cfg=62)
    pos, coef, sb = _dev(p)
    V = synth.complex_normal(np.random.default_rng(8), (p.N, 13))
    Vt = torch.from_numpy(V).cuda()
    Zo = oracle.fill(p.pos, p.freq_hz, p.coef, p.self_blocks)
    Z = harp.fill(pos, p.freq_hz, coef, sb, prec="mixed")
    X, _ = harp.solve(Z, Vt, prec="mixed")
    assert _rel(X.cpu().numpy(), oracle.solve(Zo, V)) <= 1e-10
    Xt, _ = harp.solve(None, Vt, prec="mixed", trans="T")
    assert _rel(Xt.cpu().numpy(), oracle.solve(Zo, V, trans="T")) <= 1e-10


def test_tournament_fp32_solve_within_fp32_bound(harp):
    p = synth.station()
    pos, coef, sb = _dev(p)
    Z = harp.fill(pos, p.freq_hz, coef, sb, prec="fp32")
    X, _ = harp.solve(Z, None, nrhs=p.Na, prec="fp32")
    Zo = oracle.fill(p.pos, p.freq_hz, p.coef, p.self_blocks)
    Xg = X.cpu().numpy()
    eta = np.linalg.norm(Zo @ Xg - p.V) / (np.linalg.norm(Zo) * np.linalg.norm(Xg))
    assert eta <= 1e-5 + 16 * math.sqrt(p.N) * 2.0 ** -24


@pytest.mark.parametrize("i", [0, 63])
def test_tournament_wideband_extremes(harp, i):
    """50 MHz (Nm 6, N 1536) and 350 MHz (Nm 20, N 5120): the latter's first
    panels exceed the tournament's 4096 rows and use partial pivoting."""
    p = synth.wideband()[i]
    pos, coef, sb = _dev(p)
    Z = harp.fill(pos, p.freq_hz, coef, sb, prec="mixed")
    X, info = harp.solve(Z, None, nrhs=p.Na, prec="mixed", max_iter=10)
    Zo = oracle.fill(p.pos, p.freq_hz, p.coef, p.self_blocks)
    assert _rel(X.cpu().numpy(), oracle.solve(Zo, p.V)) <= 1e-10


def test_tournament_zero_pivot_reported(harp):
    """A zero column: every candidate of that step is zero, the root reports
    the column (singular matrix) and X is not written."""
    from paper_1702_03781_gb300.harp import HarpError
    p = synth.small(40, 3, seed_cfg=63)
    pos, coef, sb = _dev(p)
    Z = harp.fill(pos, p.freq_hz, coef, sb, prec="mixed")
    Z[:, 17] = 0
    with pytest.raises(HarpError) as e:
        harp.solve(Z, None, nrhs=p.Na, prec="mixed")
    assert 1 <= e.value.status <= p.N
