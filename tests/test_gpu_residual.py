"""GPU parity of the refinement residual R = V - op(Z) X (FP64 Z and V, FP32
X) for both methods: exact integer slices on the tensor cores and the
float-float FP32-pipe kernel.

Bound: |R_ij - R*_ij| <= 2^-50 sum_k |z_ik| max_k |x_kj| + 2^-52 |V_ij|
(|z| = |re| + |im|): about 8 units of FP64 rounding of the product's scale --
what the stopping test of the refinement (tol = sqrt(N) 2^-53 against
||Z||_inf max|x_j|) needs -- plus the rounding of R itself to FP64. R* is the same expression in numpy FP64 (its own error, ~1e-17 of
that scale here, is far inside the bound) or, for small N, in long double.
A dropped digit group (~2^-7 per group) or an inexact tensor-core sum
(~2^-24) would exceed it by orders of magnitude.
"""
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
    h = Harp(0, max_N=3072, max_nrhs=256)
    assert h.residual_method() == "slices"
    yield h
    h.close()


def _cabs1(a):
    return np.abs(a.real) + np.abs(a.imag)


def _reference(Z, X, V, trans, exact):
    A = Z.T if trans == "T" else Z
    if exact:
        ld = np.longdouble
        Ar, Ai = A.real.astype(ld), A.imag.astype(ld)
        Xr, Xi = X.real.astype(ld), X.imag.astype(ld)
        Rr = V.real.astype(ld) - (Ar @ Xr - Ai @ Xi)
        Ri = V.imag.astype(ld) - (Ar @ Xi + Ai @ Xr)
        return Rr, Ri, A
    R = V - A @ X
    return R.real, R.imag, A


def _check(harp, Z, X, V, trans, method, exact=False):
    harp.set_residual(method)
    d = "cuda:0"
    R = harp.residual(torch.from_numpy(Z).to(d), torch.from_numpy(X).to(d),
                      torch.from_numpy(V).to(d), trans=trans).cpu().numpy()
    Rr, Ri, A = _reference(Z, X.astype(np.complex128), V, trans, exact)
    err = np.abs(R.real - Rr) + np.abs(R.imag - Ri)
    scale = _cabs1(A).sum(axis=1)[:, None] * _cabs1(X).max(axis=0)[None, :]
    bound = 2.0 ** -50 * scale + 2.0 ** -52 * _cabs1(V)
    ok = err <= bound
    assert ok.all(), f"{method} {trans}: worst err/bound {float(np.max(err / bound)):.3e}"
    return float(np.max(err / bound))


def _random(N, nrhs, seed):
    rng = np.random.default_rng(seed)
    Z = synth.complex_normal(rng, (N, N))
    X = synth.complex_normal(rng, (N, nrhs)).astype(np.complex64)
    V = synth.complex_normal(rng, (N, nrhs))
    return Z, X, V


@pytest.mark.parametrize("method", ["slices", "ff"])
@pytest.mark.parametrize("trans", ["N", "T"])
@pytest.mark.parametrize("N,nrhs", [(1, 1), (37, 5), (200, 3), (130, 70), (257, 129)])
def test_residual_random_shapes(harp, method, trans, N, nrhs):
    Z, X, V = _random(N, nrhs, 11 * N + nrhs)
    _check(harp, Z, X, V, trans, method, exact=True)


@pytest.mark.parametrize("method", ["slices", "ff"])
def test_residual_station_matrix(harp, method):
    """The 256-antenna station's reduced matrix against the FP32 solution of
    the port system (the first residual of the refinement), 32 columns."""
    p = synth.station()
    Z = oracle.fill(p.pos, p.freq_hz, p.coef, p.self_blocks)
    V = synth.port_rhs(p.Na, p.Nm)[:, :32]
    X = np.linalg.solve(Z.astype(np.complex64), V.astype(np.complex64)).astype(np.complex64)
    for trans in ("N", "T"):
        _check(harp, Z, X, V, trans, method)


@pytest.mark.parametrize("method", ["slices", "ff"])
def test_residual_wide_dynamic_range_zero_rows_and_columns(harp, method):
    """Rows of Z scaled by 2^[-40, 40], columns of X by 2^[-30, 30], one zero
    row of Z and one zero column of X: the per-row and per-column power-of-two
    scalings of the slices must keep every element at its own scale."""
    N, nrhs = 300, 9
    Z, X, V = _random(N, nrhs, 5)
    rng = np.random.default_rng(6)
    Z *= np.ldexp(1.0, rng.integers(-40, 41, N))[:, None]
    X = (X * np.ldexp(1.0, rng.integers(-30, 31, nrhs))[None, :]).astype(np.complex64)
    Z[17, :] = 0
    X[:, 4] = 0
    for trans in ("N", "T"):
        _check(harp, Z, X, V, trans, method, exact=True)


def test_mixed_solve_same_result_with_either_residual(harp):
    """The station's port solve refined with either residual method: both
    within 1e-10 of the FP64 oracle solution and converged to the stopping
    tolerance."""
    p = synth.station()
    d = "cuda:0"
    pos, coef, sb = (torch.from_numpy(x).to(d) for x in (p.pos, p.coef, p.self_blocks))
    Xo = oracle.solve(oracle.fill(p.pos, p.freq_hz, p.coef, p.self_blocks),
                      synth.port_rhs(p.Na, p.Nm))
    out = {}
    for method in ("slices", "ff"):
        harp.set_residual(method)
        Z = harp.fill(pos, p.freq_hz, coef, sb, prec="mixed")
        X, info = harp.solve(Z, None, nrhs=p.Na, prec="mixed")
        Xn = X.cpu().numpy()
        assert np.linalg.norm(Xn - Xo) / np.linalg.norm(Xo) <= 1e-10
        assert info["resid"] <= np.sqrt(p.N) * 2.0 ** -53
        out[method] = Xn
    harp.set_residual("slices")
    assert np.linalg.norm(out["slices"] - out["ff"]) / np.linalg.norm(out["ff"]) <= 1e-11
