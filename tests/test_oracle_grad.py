"""Pins for the oracle's position gradient of the port objective
J = sum_mn |(E^T Z^{-1} E)_mn|^2: central finite differences with
Richardson extrapolation, translation invariance, and the rotation identity
(rotating the layout equals rephasing the harmonics, Eq. 3)."""

import numpy as np
import pytest

import oracle
from paper_1702_03781_gb300 import synth


def _J(p, pos=None, coef=None):
    J, _ = oracle.port_objective_grad(p.pos if pos is None else pos, p.freq_hz,
                                      p.coef if coef is None else coef, p.self_blocks,
                                      want_grad=False)
    return J


def _problem():
    return synth.small(6, 3, P=2, Q=2, seed_cfg=11)


def test_objective_matches_explicit_solve():
    p = _problem()
    J, _ = oracle.port_objective_grad(p.pos, p.freq_hz, p.coef, p.self_blocks, want_grad=False)
    Z = oracle.fill(p.pos, p.freq_hz, p.coef, p.self_blocks)
    Pm = p.V.T @ np.linalg.solve(Z, p.V)
    assert J == pytest.approx(np.sum(np.abs(Pm) ** 2), rel=1e-12)


def test_gradient_matches_richardson_finite_differences():
    p = _problem()
    _, g = oracle.port_objective_grad(p.pos, p.freq_hz, p.coef, p.self_blocks)
    h = 1e-4
    gfd = np.zeros_like(g)
    for i in range(p.Na):
        for c in range(2):
            def jd(s):
                q = p.pos.copy()
                q[i, c] += s
                return _J(p, pos=q)
            d1 = (jd(h) - jd(-h)) / (2 * h)
            d2 = (jd(h / 2) - jd(-h / 2)) / h
            gfd[i, c] = (4 * d2 - d1) / 3  # Richardson: O(h^4)
    assert np.linalg.norm(g - gfd) / np.linalg.norm(gfd) < 1e-7


def test_gradient_central_difference_h1e4():
    """The h = 1e-4 m central difference of the synthesis workload agrees
    to 1e-6 relative along a random direction."""
    p = synth.small(10, 3, P=3, Q=2, seed_cfg=12)
    _, g = oracle.port_objective_grad(p.pos, p.freq_hz, p.coef, p.self_blocks)
    u = np.random.default_rng(4).standard_normal(g.shape)
    u /= np.linalg.norm(u)  # a step of h metres in configuration space
    h = 1e-4
    fd = (_J(p, pos=p.pos + h * u) - _J(p, pos=p.pos - h * u)) / (2 * h)
    assert abs(np.sum(g * u) - fd) / abs(fd) < 1e-6


def test_translation_invariance_of_gradient():
    """J depends on differences of positions only: sum_i dJ/dx_i = 0."""
    p = synth.small(12, 2, P=3, Q=2, seed_cfg=13)
    _, g = oracle.port_objective_grad(p.pos, p.freq_hz, p.coef, p.self_blocks)
    s = g.sum(axis=0)
    assert np.all(np.abs(s) < 1e-11 * np.abs(g).sum())


def test_rotation_identity():
    """sum_i (x_i dJ/dy_i - y_i dJ/dx_i) = dJ/dbeta, where a rotation by beta
    is the rephasing c_pq -> c_pq e^{j p beta} (Eq. 3); the right side is a
    finite difference in beta that never moves an antenna."""
    p = _problem()
    _, g = oracle.port_objective_grad(p.pos, p.freq_hz, p.coef, p.self_blocks)
    lhs = np.sum(p.pos[:, 0] * g[:, 1] - p.pos[:, 1] * g[:, 0])
    P = p.P
    pp = np.arange(-P, P + 1)

    def jb(b):
        return _J(p, coef=p.coef * np.exp(1j * pp * b)[None, None, :, None])
    h = 1e-4
    d1 = (jb(h) - jb(-h)) / (2 * h)
    d2 = (jb(h / 2) - jb(-h / 2)) / h
    rhs = (4 * d2 - d1) / 3
    assert lhs == pytest.approx(rhs, rel=1e-7, abs=1e-9 * np.abs(g).sum())


def test_adjoint_pieces_agree_with_direct_formula():
    """grad_from_adjoint with a hand-made Lambda reproduces the contraction
    -2 Re sum_ij G_ij dZ_ij/dx where dZ/dx is a finite difference of the
    fill (only the pair blocks of the moved antenna change)."""
    p = synth.small(5, 2, P=2, Q=2, seed_cfg=14)
    rng = np.random.default_rng(9)
    Lam = synth.complex_normal(rng, (p.N, 3))
    X = synth.complex_normal(rng, (p.N, 3))
    g = oracle.grad_from_adjoint(p.pos, p.freq_hz, p.coef, Lam, X)
    G = Lam @ X.T
    h = 1e-5
    for i in range(p.Na):
        for c in range(2):
            q1, q2 = p.pos.copy(), p.pos.copy()
            q1[i, c] += h
            q2[i, c] -= h
            dZ = (oracle.fill(q1, p.freq_hz, p.coef, p.self_blocks)
                  - oracle.fill(q2, p.freq_hz, p.coef, p.self_blocks)) / (2 * h)
            expect = -2 * np.real(np.sum(G * dZ))
            assert g[i, c] == pytest.approx(expect, rel=1e-6, abs=1e-8)


def _Jimp(p, pos=None):
    J, _ = oracle.port_impedance_objective_grad(p.pos if pos is None else pos, p.freq_hz,
                                                p.coef, p.self_blocks, want_grad=False)
    return J


def test_impedance_objective_matches_library_inverse():
    """The impedance reading J = sum |(E^T Z^{-1} E)^{-1}|^2, against numpy's
    LAPACK solve and inverse on the oracle's Z."""
    p = _problem()
    J, _ = oracle.port_impedance_objective_grad(p.pos, p.freq_hz, p.coef, p.self_blocks,
                                                want_grad=False)
    Z = oracle.fill(p.pos, p.freq_hz, p.coef, p.self_blocks)
    Zp = np.linalg.inv(p.V.T @ np.linalg.solve(Z, p.V))
    assert J == pytest.approx(np.sum(np.abs(Zp) ** 2), rel=1e-11)


def test_impedance_gradient_matches_richardson_finite_differences():
    p = _problem()
    _, g = oracle.port_impedance_objective_grad(p.pos, p.freq_hz, p.coef, p.self_blocks)
    h = 1e-4
    gfd = np.zeros_like(g)
    for i in range(p.Na):
        for c in range(2):
            def jd(s):
                q = p.pos.copy()
                q[i, c] += s
                return _Jimp(p, pos=q)
            d1 = (jd(h) - jd(-h)) / (2 * h)
            d2 = (jd(h / 2) - jd(-h / 2)) / h
            gfd[i, c] = (4 * d2 - d1) / 3
    assert np.linalg.norm(g - gfd) / np.linalg.norm(gfd) < 1e-7


def test_impedance_gradient_translation_invariance():
    p = synth.small(12, 2, P=3, Q=2, seed_cfg=13)
    _, g = oracle.port_impedance_objective_grad(p.pos, p.freq_hz, p.coef, p.self_blocks)
    assert np.all(np.abs(g.sum(axis=0)) < 1e-11 * np.abs(g).sum())
