"""GPU parity of the FP32 factorisation with the other pivot rules, through
the C ABI against the FP64 CPU oracle:
  * tournament pivoting (the communication-avoiding LU panel);
  * pivoting restricted to each panel's diagonal block, whose factors the
    refinement checks (a zero pivot or a stalled refinement redoes the
    factorisation with partial pivoting).

Both factor the same matrix with another row order, so the refined solution
must meet the same bar as with partial pivoting: relative Frobenius error
<= 1e-10 against the oracle's X, for the port right-hand sides, general
right-hand sides and the transposed solve. The tournament panel applies to
panels of up to 4096 rows (16 CTAs of at most 256 rows), which covers every
panel of the station; larger ones use partial pivoting, which the
5120-unknown wideband case exercises. The FP32 mode keeps the backward error
bound stated in test_gpu_edge.py (the block rule uses partial pivoting
there, having no refinement to check it).
"""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_1702_03781_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", params=["tournament", "block"])
def harp(request):
    from paper_1702_03781_gb300 import build
    build.build()
    from paper_1702_03781_gb300.harp import Harp
    h = Harp(0, max_N=5120, max_nrhs=256)
    h.set_pivot(request.param)
    yield h
    h.close()


def _dev(p):
    d = "cuda:0"
    return (torch.from_numpy(p.pos).to(d), torch.from_numpy(p.coef).to(d),
            torch.from_numpy(p.self_blocks).to(d))


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_pivot_option_round_trip(harp):
    rule = harp.pivot_rule()
    assert rule in ("tournament", "block")
    harp.set_pivot("partial")
    assert harp.pivot_rule() == "partial"
    harp.set_pivot(rule)
    with pytest.raises(KeyError):
        harp.set_pivot("rook")


@pytest.mark.parametrize("mk", [lambda: synth.tiny(), lambda: synth.small(37, 5, P=3, Q=2),
                                lambda: synth.small(70, 3, P=2, Q=4, seed_cfg=21),
                                lambda: synth.small(150, 9, P=3, Q=3, seed_cfg=61),
                                lambda: synth.station()])
def test_mixed_solve_matches_oracle(harp, mk):
    p = mk()
    pos, coef, sb = _dev(p)
    Z = harp.fill(pos, p.freq_hz, coef, sb, prec="mixed")
    X, info = harp.solve(Z, None, nrhs=p.Na, prec="mixed", max_iter=10)
    Zo = oracle.fill(p.pos, p.freq_hz, p.coef, p.self_blocks)
    assert _rel(X.cpu().numpy(), oracle.solve(Zo, p.V)) <= 1e-10
    assert info["resid"] <= math.sqrt(p.N) * 2.0 ** -53


def test_general_rhs_and_transpose(harp):
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


def test_fp32_solve_within_fp32_bound(harp):
    p = synth.station()
    pos, coef, sb = _dev(p)
    Z = harp.fill(pos, p.freq_hz, coef, sb, prec="fp32")
    X, _ = harp.solve(Z, None, nrhs=p.Na, prec="fp32")
    Zo = oracle.fill(p.pos, p.freq_hz, p.coef, p.self_blocks)
    Xg = X.cpu().numpy()
    eta = np.linalg.norm(Zo @ Xg - p.V) / (np.linalg.norm(Zo) * np.linalg.norm(Xg))
    assert eta <= 1e-5 + 16 * math.sqrt(p.N) * 2.0 ** -24


@pytest.mark.parametrize("i", [0, 63])
def test_wideband_extremes(harp, i):
    """50 MHz (Nm 6, N 1536) and 350 MHz (Nm 20, N 5120): the latter's first
    panels exceed the tournament's 4096 rows and use partial pivoting."""
    p = synth.wideband()[i]
    pos, coef, sb = _dev(p)
    Z = harp.fill(pos, p.freq_hz, coef, sb, prec="mixed")
    X, info = harp.solve(Z, None, nrhs=p.Na, prec="mixed", max_iter=10)
    Zo = oracle.fill(p.pos, p.freq_hz, p.coef, p.self_blocks)
    assert _rel(X.cpu().numpy(), oracle.solve(Zo, p.V)) <= 1e-10


def test_zero_pivot_reported(harp):
    """A zero column: every candidate of that step is zero, the matrix is
    singular, and the column is reported (the block rule's retry with
    partial pivoting meets the same zero)."""
    from paper_1702_03781_gb300.harp import HarpError
    p = synth.small(40, 3, seed_cfg=63)
    pos, coef, sb = _dev(p)
    Z = harp.fill(pos, p.freq_hz, coef, sb, prec="mixed")
    Z[:, 17] = 0
    with pytest.raises(HarpError) as e:
        harp.solve(Z, None, nrhs=p.Na, prec="mixed")
    assert 1 <= e.value.status <= p.N


def _restricted_case(harp, scale):
    """A problem whose first diagonal block (rows and columns 0..63) is
    scaled by `scale` in both Z and the context's Z64, and its FP64 solution
    from numpy on the same Z64."""
    p = synth.small(110, 7, P=2, Q=2, seed_cfg=64)
    pos, coef, sb = _dev(p)
    Z = harp.fill(pos, p.freq_hz, coef, sb, prec="mixed")
    Z64 = harp.z64(p.N)
    Z64[:64, :64] *= scale
    Z[:64, :64] = Z64[:64, :64].to(torch.complex64)
    Zn = Z64.cpu().numpy()
    return p, Z, np.linalg.solve(Zn, p.V)


def test_block_rule_falls_back_on_a_zero_block_pivot(harp):
    """The first diagonal block is zero, the matrix is not singular: the
    block rule meets a zero pivot, refactors with partial pivoting and
    solves."""
    if harp.pivot_rule() != "block":
        pytest.skip("block rule only")
    before = harp.pivot_fallbacks()
    p, Z, Xr = _restricted_case(harp, 0.0)
    X, info = harp.solve(Z, None, nrhs=p.Na, prec="mixed", max_iter=10)
    assert harp.pivot_fallbacks() == before + 1
    assert _rel(X.cpu().numpy(), Xr) <= 1e-10


def test_block_rule_falls_back_when_the_refinement_stalls(harp):
    """A tiny first diagonal block makes the restricted factors useless
    (L21 = A21 U11^-1 grows like 1 / scale): the refinement stops
    contracting, the factorisation is redone with partial pivoting and the
    solution meets the tolerance."""
    if harp.pivot_rule() != "block":
        pytest.skip("block rule only")
    before = harp.pivot_fallbacks()
    p, Z, Xr = _restricted_case(harp, 1e-5)
    X, info = harp.solve(Z, None, nrhs=p.Na, prec="mixed", max_iter=10)
    assert harp.pivot_fallbacks() == before + 1
    assert _rel(X.cpu().numpy(), Xr) <= 1e-10
