"""Pins for the oracle's LU and substitution (the direct solve of Section
II-B) and the port objective: LAPACK (numpy), closed forms, structure."""
import numpy as np
import pytest

import oracle
from paper_1702_03781_gb300 import synth


def _rand(N, seed, dd=0.0):
    rng = np.random.default_rng(seed)
    A = synth.complex_normal(rng, (N, N))
    A += dd * np.eye(N)
    return np.asfortranarray(A)


@pytest.mark.parametrize("N,nrhs", [(1, 1), (2, 3), (7, 2), (64, 16), (193, 5)])
def test_solve_matches_lapack(N, nrhs):
    A = _rand(N, N)
    B = synth.complex_normal(np.random.default_rng(N + 1), (N, nrhs))
    X = oracle.solve(A, B)
    Xl = np.linalg.solve(A, B)
    cond = np.linalg.cond(A)
    assert oracle.relerr(X, Xl) < max(1e-14, 50 * cond * 2.2e-16)


@pytest.mark.parametrize("N", [5, 64, 150])
def test_transposed_solve_matches_lapack(N):
    A = _rand(N, 10 + N)
    B = synth.complex_normal(np.random.default_rng(N), (N, 4))
    X = oracle.solve(A, B, trans="T")
    Xl = np.linalg.solve(A.T, B)
    assert oracle.relerr(X, Xl) < 50 * np.linalg.cond(A) * 2.2e-16


def test_cramer_2x2():
    A = np.array([[1 + 2j, 3 - 1j], [-2 + 0.5j, 4 + 4j]], order="F")
    b = np.array([[1 - 1j], [2 + 3j]])
    det = A[0, 0] * A[1, 1] - A[0, 1] * A[1, 0]
    x0 = (b[0, 0] * A[1, 1] - A[0, 1] * b[1, 0]) / det
    x1 = (A[0, 0] * b[1, 0] - b[0, 0] * A[1, 0]) / det
    X = oracle.solve(A, b)
    assert X[0, 0] == pytest.approx(x0, rel=1e-15)
    assert X[1, 0] == pytest.approx(x1, rel=1e-15)


def test_partial_pivoting_choice():
    """The pivot of each column is the entry of largest modulus."""
    A = np.array([[1e-3, 1, 2], [3 + 4j, 1, 0], [-4, 2j, 1]], dtype=np.complex128, order="F")
    LU, ipiv, info = oracle.lu(A)
    assert info == 0
    assert ipiv[0] == 1  # |3+4j| = 5 beats |-4| = 4 and 1e-3
    L = np.tril(LU, -1) + np.eye(3)
    U = np.triu(LU)
    assert np.all(np.abs(np.tril(LU, -1)) <= 1 + 1e-15)
    PA = A.copy()
    for k, p in enumerate(ipiv):
        PA[[k, p]] = PA[[p, k]]
    np.testing.assert_allclose(L @ U, PA, rtol=1e-15, atol=1e-15)


def test_lu_reconstructs_permuted_matrix():
    A = _rand(97, 3)
    LU, ipiv, info = oracle.lu(A)
    assert info == 0
    L = np.tril(LU, -1) + np.eye(97)
    U = np.triu(LU)
    PA = A.copy()
    for k, p in enumerate(ipiv):
        PA[[k, p]] = PA[[p, k]]
    assert oracle.relerr(L @ U, PA) < 1e-14
    assert np.all(np.abs(np.tril(LU, -1)) <= 1.0 + 1e-15)


def test_zero_pivot_reported():
    A = _rand(6, 4)
    A[:, 2] = 0.0
    _, _, info = oracle.lu(A)
    assert info == 3
    with pytest.raises(np.linalg.LinAlgError):
        oracle.solve(A, np.ones((6, 1)))


def test_block_diagonal_when_no_coupling():
    """All HARP coefficients zero: Z is block diagonal and X splits into Na
    independent Nm x Nm solves of the self blocks."""
    p = synth.small(9, 4)
    Z = oracle.fill(p.pos, p.freq_hz, np.zeros_like(p.coef), p.self_blocks)
    X = oracle.solve(Z, p.V)
    Xb = np.zeros_like(X)
    for a in range(9):
        sl = slice(4 * a, 4 * a + 4)
        Xb[sl, :] = np.linalg.solve(p.self_blocks[a], p.V[sl, :])
    assert oracle.relerr(X, Xb) < 1e-14


def test_residual_bound_station_shaped():
    """A filled HARP system: residual ||ZX - V|| / (||Z|| ||X||) within a
    small multiple of N eps, and agreement with LAPACK within cond * eps."""
    p = synth.small(40, 5, P=3, Q=3)
    Z = oracle.fill(p.pos, p.freq_hz, p.coef, p.self_blocks)
    X = oracle.solve(Z, p.V)
    N = Z.shape[0]
    res = np.linalg.norm(Z @ X - p.V) / (np.linalg.norm(Z) * np.linalg.norm(X))
    assert res < 10 * N * 2.2e-16
    assert oracle.relerr(X, np.linalg.solve(Z, p.V)) < 50 * np.linalg.cond(Z) * 2.2e-16


def test_tiny_config_solve():
    """16 antennas x 4 MBFs, 16 port RHS: oracle against LAPACK."""
    p = synth.tiny()
    Z = oracle.fill(p.pos, p.freq_hz, p.coef, p.self_blocks)
    X = oracle.solve(Z, p.V)
    assert X.shape == (64, 16)
    assert oracle.relerr(X, np.linalg.solve(Z, p.V)) < 1e-12


def test_port_objective():
    """P = E^T X picks row m*Nm of each column; J = sum |P|^2."""
    Na, Nm = 5, 3
    X = synth.complex_normal(np.random.default_rng(1), (Na * Nm, Na))
    E = synth.port_rhs(Na, Nm)
    J, Pm = oracle.port_objective(X, Na, Nm)
    np.testing.assert_array_equal(Pm, E.T @ X)
    assert J == pytest.approx(np.sum(np.abs(E.T @ X) ** 2), rel=1e-15)


def test_port_rhs_selects_mbf0():
    V = synth.port_rhs(4, 3)
    assert V.shape == (12, 4)
    assert np.array_equal(np.argwhere(V != 0), np.array([[0, 0], [3, 1], [6, 2], [9, 3]]))
