"""GPU parity for the exported precision modes, the method's degenerate
shapes and the documented statuses, through the C ABI against the FP64 CPU
oracle (and, for P = Q = 0, against the closed form directly).

Tolerances (stated here, derived from the arithmetic):
  * FP32 solve (HARP_FP32, no refinement): the matrix is the FP32 fill, whose
    relative error is within the 1e-5 fill tolerance, factored in FP32 with
    three-term TF32 products (about 3 * 2^-24 per product). The normwise
    backward error against the oracle's matrix,
        ||Zo X - V||_F / (||Zo||_F ||X||_F),
    is therefore bounded by 1e-5 + 16 sqrt(N) 2^-24 (fill error plus an LU
    term that grows like sqrt(N) for random rounding), and the forward error
    by cond_2(Zo) times that bound.
  * refined solutions (FP64, mixed 3xTF32, mixed TF32 where it converges):
    relative Frobenius error <= 1e-10 against the oracle's X.
  * a solve that stops without meeting the tolerance (HARP_E_NOCONV) returns
    the iterate with the smallest backward error seen: the reported
    resid_out must equal the zcgesv column test of the returned X evaluated
    against the oracle's matrix, to 1e-3 relative (the two differ only by the
    FP64 rounding of the residual, far below the stalled error).
  * the P = Q = 0 fill: every mutual entry equals c_00 e^{-jkr} within
    1e-13 of max |c_00| (FP64 on both sides; the phase kr, up to ~50 rad
    here, carries a few ulp of argument reduction, ~1e-14).
"""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_1702_03781_gb300 import synth

pytestmark = pytest.mark.gpu

C0 = 299792458.0


@pytest.fixture(scope="module")
def harp():
    from paper_1702_03781_gb300 import build
    build.build()
    from paper_1702_03781_gb300.harp import Harp
    h = Harp(0, max_N=3072, max_nrhs=256)
    yield h
    h.close()


def _dev(p):
    d = "cuda:0"
    return (torch.from_numpy(p.pos).to(d), torch.from_numpy(p.coef).to(d),
            torch.from_numpy(p.self_blocks).to(d))


def _np(t):
    return t.detach().cpu().numpy()


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _zcgesv_test(Z, X, V):
    """max over columns of max_i |R_ij| / (||Z||_inf max_i |X_ij|), with
    |z| = |re| + |im| and R = V - Z X (the stopping test of the refinement)."""
    a1 = lambda z: np.abs(z.real) + np.abs(z.imag)  # noqa: E731
    R = V - Z @ X
    znorm = np.max(np.sum(a1(Z), axis=1))
    return float(np.max(np.max(a1(R), axis=0) / (znorm * np.max(a1(X), axis=0))))


# ---- HARP_FP32: FP32 fill and three-term TF32 LU, no refinement ----------

@pytest.mark.parametrize("mk", [lambda: synth.tiny(), lambda: synth.small(37, 5, P=3, Q=2),
                                lambda: synth.station()])
def test_fp32_solve_within_fp32_bounds(harp, mk):
    p = mk()
    pos, coef, sb = _dev(p)
    Z = harp.fill(pos, p.freq_hz, coef, sb, prec="fp32")
    X, info = harp.solve(Z, None, nrhs=p.Na, prec="fp32")
    assert info["iters"] == 0 and info["resid"] == -1.0
    Zo = oracle.fill(p.pos, p.freq_hz, p.coef, p.self_blocks)
    Xg = _np(X)
    bound = 1e-5 + 16 * math.sqrt(p.N) * 2.0 ** -24
    eta = np.linalg.norm(Zo @ Xg - p.V) / (np.linalg.norm(Zo) * np.linalg.norm(Xg))
    assert eta <= bound
    if p.N <= 512:
        cond = np.linalg.cond(Zo)
        assert _rel(Xg, oracle.solve(Zo, p.V)) <= cond * bound
    # and far from the refined accuracy: the mode really stops at FP32 level
    assert eta >= 1e-12


# ---- HARP_MIXED_TF32: single-term TF32 products with refinement ----------

def test_mixed_tf32_converges_on_a_well_conditioned_case(harp):
    p = synth.tiny()
    pos, coef, sb = _dev(p)
    Zo = oracle.fill(p.pos, p.freq_hz, p.coef, p.self_blocks)
    # the regime where TF32 refinement contracts: the error shrinks by about
    # cond * 2^-11 per correction (0.19 here)
    assert np.linalg.cond(Zo) * 2.0 ** -11 < 0.5
    Z = harp.fill(pos, p.freq_hz, coef, sb, prec="mixed_tf32")
    X, info = harp.solve(Z, None, nrhs=p.Na, prec="mixed_tf32", max_iter=30)
    assert info["status"] == 0
    assert _rel(_np(X), oracle.solve(Zo, p.V)) <= 1e-10


def test_mixed_tf32_station_reports_noconv_with_best_iterate(harp):
    """At the station cond_2 ~ 7.5e4, so cond * 2^-11 >> 1: single-term TF32
    factors do not make refinement contract (the forward error of the first
    solution is already of the order of the solution itself). The call must
    say so and return the iterate of smallest backward error, whose error it
    reports."""
    from paper_1702_03781_gb300.harp import HARP_E_NOCONV
    p = synth.station()
    pos, coef, sb = _dev(p)
    Z = harp.fill(pos, p.freq_hz, coef, sb, prec="mixed_tf32")
    X, info = harp.solve(Z, None, nrhs=p.Na, prec="mixed_tf32", max_iter=10,
                         allow_noconv=True)
    tol = math.sqrt(p.N) * 2.0 ** -53
    assert info["status"] == HARP_E_NOCONV
    assert info["iters"] == 10 and info["resid"] > tol
    Zo = oracle.fill(p.pos, p.freq_hz, p.coef, p.self_blocks)
    Xg = _np(X)
    assert np.all(np.isfinite(Xg))
    got = _zcgesv_test(Zo, Xg, p.V)
    assert got == pytest.approx(info["resid"], rel=1e-3)
    assert info["resid"] < 1.0


def test_max_iter_zero_returns_the_first_solution_and_noconv(harp):
    from paper_1702_03781_gb300.harp import HARP_E_NOCONV
    p = synth.tiny()
    pos, coef, sb = _dev(p)
    Z = harp.fill(pos, p.freq_hz, coef, sb, prec="mixed")
    X, info = harp.solve(Z, None, nrhs=p.Na, prec="mixed", max_iter=0, allow_noconv=True)
    assert info["status"] == HARP_E_NOCONV and info["iters"] == 0
    Zo = oracle.fill(p.pos, p.freq_hz, p.coef, p.self_blocks)
    assert _zcgesv_test(Zo, _np(X), p.V) == pytest.approx(info["resid"], rel=1e-3)
    # the same context then refines normally
    X, info = harp.solve(Z, None, nrhs=p.Na, prec="mixed", max_iter=10)
    assert _rel(_np(X), oracle.solve(Zo, p.V)) <= 1e-10


# ---- degenerate shapes of the method --------------------------------------

@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("Na,Nm,P,Q", [(1, 5, 2, 2), (1, 1, 0, 0), (40, 1, 2, 2),
                                       (30, 3, 0, 0), (2, 4, 1, 1)])
def test_degenerate_shapes_fill_and_solve(harp, prec, Na, Nm, P, Q):
    """One antenna (no pairs: Z is the self block), one MBF per antenna,
    P = Q = 0 (a single basis term), two antennas."""
    p = synth.small(Na, Nm, P=P, Q=Q, seed_cfg=51)
    pos, coef, sb = _dev(p)
    Zo = oracle.fill(p.pos, p.freq_hz, p.coef, p.self_blocks)
    Z = harp.fill(pos, p.freq_hz, coef, sb, prec=prec)
    if prec == "fp64":
        assert np.max(np.abs(_np(Z) - Zo)) <= 1e-13 * np.max(np.abs(Zo))
    else:
        assert np.max(np.abs(harp.z64(p.N).cpu().numpy() - Zo)) <= 1e-13 * np.max(np.abs(Zo))
    X, info = harp.solve(Z, None, nrhs=p.Na, prec=prec, max_iter=10)
    assert _rel(_np(X), oracle.solve(Zo, p.V)) <= 1e-10


def test_p_q_zero_fill_is_the_closed_form(harp):
    """P = Q = 0: Eq. 3 keeps the single term c_00, so Eq. 4 gives
    Z^{mn}_TS = c_00^{TS} e^{-jkr}, computed here in numpy from the
    positions alone."""
    p = synth.small(30, 3, P=0, Q=0, seed_cfg=52)
    pos, coef, sb = _dev(p)
    Z = _np(harp.fill(pos, p.freq_hz, coef, sb, prec="fp64"))
    k = 2 * math.pi * p.freq_hz / C0
    c00 = p.coef[:, :, 0, 0]  # [T, S]
    Nm = p.Nm
    for m in range(p.Na):
        for n in range(p.Na):
            blk = Z[m * Nm:(m + 1) * Nm, n * Nm:(n + 1) * Nm]
            if m == n:
                assert np.array_equal(blk, p.self_blocks[m])
                continue
            r = math.hypot(*(p.pos[m] - p.pos[n]))
            ref = c00 * np.exp(-1j * k * r)
            assert np.max(np.abs(blk - ref)) <= 1e-13 * np.max(np.abs(c00))


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_single_right_hand_side(harp, prec):
    p = synth.small(30, 4, P=2, Q=2, seed_cfg=53)
    pos, coef, sb = _dev(p)
    V = synth.complex_normal(np.random.default_rng(5), (p.N, 1))
    Vt = torch.from_numpy(V).cuda()
    Zo = oracle.fill(p.pos, p.freq_hz, p.coef, p.self_blocks)
    Z = harp.fill(pos, p.freq_hz, coef, sb, prec=prec)
    X, _ = harp.solve(Z, Vt, prec=prec)
    assert _rel(_np(X), oracle.solve(Zo, V)) <= 1e-10
    Xt, _ = harp.solve(None, Vt, prec=prec, trans="T")
    assert _rel(_np(Xt), oracle.solve(Zo, V, trans="T")) <= 1e-10


# ---- statuses made on the host --------------------------------------------

@pytest.mark.parametrize("where", ["pos", "coef", "self"])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_nonfinite_input_reported(harp, where, prec):
    """A NaN in the positions, the coefficients or a self block: the fill
    leaves HARP_E_NONFINITE pending; the next solve returns it, and the
    context keeps working afterwards."""
    from paper_1702_03781_gb300.harp import HarpError, HARP_E_NONFINITE
    p = synth.small(12, 3, P=2, Q=1, seed_cfg=54)
    pos, coef, sb = _dev(p)
    bad = {"pos": pos.clone(), "coef": coef.clone(), "self": sb.clone()}[where]
    if where == "pos":
        bad[3, 1] = float("nan")
    else:
        bad.view(-1)[5] = complex(float("nan"), 0.0)
    args = {"pos": pos, "coef": coef, "self": sb}
    args[where] = bad
    Z = harp.fill(args["pos"], p.freq_hz, args["coef"], args["self"], prec=prec)
    with pytest.raises(HarpError) as e:
        harp.solve(Z, None, nrhs=p.Na, prec=prec)
    assert e.value.status == HARP_E_NONFINITE
    harp.fill(args["pos"], p.freq_hz, args["coef"], args["self"], prec=prec)
    with pytest.raises(HarpError) as e:
        harp.sync()
    assert e.value.status == HARP_E_NONFINITE
    Z = harp.fill(pos, p.freq_hz, coef, sb, prec=prec)
    X, _ = harp.solve(Z, None, nrhs=p.Na, prec=prec)
    Zo = oracle.fill(p.pos, p.freq_hz, p.coef, p.self_blocks)
    assert _rel(_np(X), oracle.solve(Zo, p.V)) <= 1e-10


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_nonfinite_matrix_or_rhs_reported(harp, prec):
    """A NaN in a caller's matrix is caught as the solve copies it in. A NaN
    right-hand side: the mixed refinement's stopping test returns the status;
    the FP64 solve, which does not synchronise after its substitutions,
    leaves it pending for harp_ctx_sync."""
    from paper_1702_03781_gb300.harp import HarpError, HARP_E_NONFINITE
    p = synth.small(12, 3, P=2, Q=1, seed_cfg=55)
    pos, coef, sb = _dev(p)
    Z = harp.fill(pos, p.freq_hz, coef, sb, prec=prec)
    Zb = Z.clone()
    Zb[4, 7] = complex(float("inf"), 0.0)
    with pytest.raises(HarpError) as e:
        harp.solve(Zb, None, nrhs=p.Na, prec=prec)
    assert e.value.status == HARP_E_NONFINITE
    V = torch.ones((p.N, 2), dtype=torch.complex128, device="cuda:0")
    V[3, 1] = complex(float("nan"), 0.0)
    if prec == "fp64":
        harp.solve(Z, V, prec=prec)
        with pytest.raises(HarpError) as e:
            harp.sync()
    else:
        with pytest.raises(HarpError) as e:
            harp.solve(Z, V, prec=prec)
    assert e.value.status == HARP_E_NONFINITE
    harp.sync()
