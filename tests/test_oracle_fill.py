"""Pins for the oracle's HARP fill (Eq. 1, 3, 4), independent of the oracle.

Every expected value here comes from a closed form, a symmetry of the
model, or a hand derivation -- never from the oracle itself or from the
CUDA path.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1702_03781_gb300 import synth

C0 = 299_792_458.0
F = 110e6
K = 2 * math.pi * F / C0


def _coef_zero(Nm, P, Q):
    return np.zeros((Nm, Nm, 2 * P + 1, Q + 1), dtype=np.complex128)


def _blocks(Z, Na, Nm):
    """(Na, Na, Nm, Nm) view: [m, n, T, S] = Z[m*Nm+T, n*Nm+S]."""
    return np.asarray(Z).reshape(Na, Nm, Na, Nm).transpose(0, 2, 1, 3)


def _pairs(Na):
    return [(m, n) for m in range(Na) for n in range(Na) if m != n]


def test_wavenumber():
    # k = 2 pi f / c0 at 110 MHz (lambda = 2.72539 m)
    assert oracle.wavenumber(F) == pytest.approx(2 * math.pi / (C0 / F), rel=1e-15)
    assert C0 / F == pytest.approx(2.7253859818, rel=1e-9)


def test_phase_only_closed_form():
    """P = Q = 0, c_00 = 1: every mutual entry is e^{-jkr} (Eq. 3-4)."""
    p = synth.small(7, 2, P=0, Q=0)
    c = _coef_zero(2, 0, 0)
    c[:, :, 0, 0] = 1.0
    Z = oracle.fill(p.pos, F, c, p.self_blocks)
    B = _blocks(Z, 7, 2)
    for m, n in _pairs(7):
        r = np.hypot(*(p.pos[m] - p.pos[n]))
        np.testing.assert_allclose(B[m, n], np.full((2, 2), np.exp(-1j * K * r)), rtol=2e-15, atol=0)


def test_green_function_closed_form():
    """c_01 = 1 (q = 1, d = 1/r): the free-space kernel e^{-jkr}/r."""
    p = synth.small(6, 1, P=0, Q=1)
    c = _coef_zero(1, 0, 1)
    c[0, 0, 0, 1] = 1.0
    Z = oracle.fill(p.pos, F, c, p.self_blocks)
    for m, n in _pairs(6):
        r = np.hypot(*(p.pos[m] - p.pos[n]))
        assert Z[m, n] == pytest.approx(np.exp(-1j * K * r) / r, rel=2e-15)


def test_original_change_of_variables():
    """dvar = 2 is the original model's d = 1/r^2: c_01 = 1 gives e^{-jkr}/r^2."""
    p = synth.small(5, 1, P=0, Q=1)
    c = _coef_zero(1, 0, 1)
    c[0, 0, 0, 1] = 1.0
    Z = oracle.fill(p.pos, F, c, p.self_blocks, dvar=2)
    for m, n in _pairs(5):
        r = np.hypot(*(p.pos[m] - p.pos[n]))
        assert Z[m, n] == pytest.approx(np.exp(-1j * K * r) / r ** 2, rel=2e-15)


@pytest.mark.parametrize("p_h", [-3, -1, 1, 2, 4])
def test_single_harmonic_on_axes(p_h):
    """Antennas on the axes around a source at the origin: alpha is
    0, pi/2, pi, -pi/2 exactly, so e^{j p alpha} = 1, j^p, (-1)^p, (-j)^p."""
    D = 3.0
    pos = np.array([[0, 0], [D, 0], [0, D], [-D, 0], [0, -D]], dtype=np.float64)
    P = 4
    c = _coef_zero(1, P, 0)
    c[0, 0, p_h + P, 0] = 1.0
    sb = np.ones((5, 1, 1), dtype=np.complex128)
    Z = oracle.fill(pos, F, c, sb)
    ph = np.exp(-1j * K * D)
    expect = {1: 1.0, 2: 1j ** p_h, 3: (-1.0) ** p_h, 4: (-1j) ** p_h}
    for m, e in expect.items():
        assert Z[m, 0] == pytest.approx(e * ph, rel=1e-15, abs=1e-15)


def test_two_antennas_hand_derivation():
    """Na = 2 at (0,0) and (D,0). Block (1,0) sees alpha = 0 and block (0,1)
    sees alpha = pi, so Z^{10}_TS = e^{-jkD} sum_p sum_q c_pq D^-q and
    Z^{01}_TS = e^{-jkD} sum_p (-1)^p sum_q c_pq D^-q."""
    D, Nm, P, Q = 2.5, 3, 2, 3
    c = synth.harp_coefficients(Nm, P, Q, 77)
    pos = np.array([[0.0, 0.0], [D, 0.0]])
    sb = synth.self_blocks(2, Nm, 78)
    Z = oracle.fill(pos, F, c, sb)
    dq = D ** -np.arange(Q + 1.0)
    sgn = (-1.0) ** np.arange(-P, P + 1)
    ph = np.exp(-1j * K * D)
    Z10 = ph * np.einsum("tspq,q->ts", c, dq)
    Z01 = ph * np.einsum("tspq,p,q->ts", c, sgn, dq)
    np.testing.assert_allclose(Z[Nm:, :Nm], Z10, rtol=1e-14, atol=1e-15)
    np.testing.assert_allclose(Z[:Nm, Nm:], Z01, rtol=1e-14, atol=1e-15)


def test_self_blocks_copied_bit_exact():
    p = synth.small(9, 3)
    Z = oracle.fill(p.pos, F, p.coef, p.self_blocks)
    B = _blocks(Z, 9, 3)
    for a in range(9):
        assert np.array_equal(B[a, a], p.self_blocks[a])
    # one shared block (identical antennas)
    Z2 = oracle.fill(p.pos, F, p.coef, p.self_blocks[4])
    B2 = _blocks(Z2, 9, 3)
    for a in range(9):
        assert np.array_equal(B2[a, a], p.self_blocks[4])
    # off-diagonal blocks do not depend on the self blocks
    mask = np.kron(1 - np.eye(9), np.ones((3, 3))).astype(bool)
    assert np.array_equal(Z[mask], Z2[mask])


def test_translation_invariance():
    p = synth.small(12, 3, P=3, Q=3)
    Z = oracle.fill(p.pos, F, p.coef, p.self_blocks)
    Zt = oracle.fill(p.pos + np.array([13.25, -7.5]), F, p.coef, p.self_blocks)
    assert oracle.relerr(Zt, Z) < 1e-14


@pytest.mark.parametrize("beta", [0.3, 1.7, -2.4])
def test_rotation_covariance(beta):
    """Rotating the layout by beta equals rephasing c_pq by e^{j p beta}."""
    p = synth.small(10, 2, P=4, Q=2)
    R = np.array([[math.cos(beta), -math.sin(beta)], [math.sin(beta), math.cos(beta)]])
    Zrot = oracle.fill(p.pos @ R.T, F, p.coef, p.self_blocks)
    ph = np.exp(1j * np.arange(-4, 5) * beta)
    Zc = oracle.fill(p.pos, F, p.coef * ph[None, None, :, None], p.self_blocks)
    assert oracle.relerr(Zrot, Zc) < 1e-13


def test_relabelling_permutes_blocks_exactly():
    p = synth.small(8, 3)
    perm = np.random.default_rng(5).permutation(8)
    Z = oracle.fill(p.pos, F, p.coef, p.self_blocks)
    Zp = oracle.fill(p.pos[perm], F, p.coef, p.self_blocks[perm])
    B, Bp = _blocks(Z, 8, 3), _blocks(Zp, 8, 3)
    for m in range(8):
        for n in range(8):
            assert np.array_equal(Bp[m, n], B[perm[m], perm[n]])


def test_swap_symmetry():
    """alpha_nm = alpha_mn + pi, so block (n,m) equals block (m,n) computed
    with c_pq (-1)^p."""
    p = synth.small(9, 2, P=3, Q=2)
    Z = oracle.fill(p.pos, F, p.coef, p.self_blocks)
    sgn = (-1.0) ** np.arange(-3, 4)
    Zs = oracle.fill(p.pos, F, p.coef * sgn[None, None, :, None], p.self_blocks)
    B, Bs = _blocks(Z, 9, 2), _blocks(Zs, 9, 2)
    for m, n in _pairs(9):
        np.testing.assert_allclose(B[n, m], Bs[m, n], rtol=1e-13, atol=1e-14)


def test_reciprocity():
    """With c^{ST}_pq = (-1)^p c^{TS}_pq and symmetric self blocks, Z = Z^T."""
    Nm, P, Q = 3, 3, 2
    p = synth.small(8, Nm, P=P, Q=Q)
    c = p.coef.copy()
    sgn = (-1.0) ** np.arange(-P, P + 1)
    for T in range(Nm):
        for S in range(T + 1, Nm):
            c[S, T] = c[T, S] * sgn[:, None]
        c[T, T] = 0.5 * (c[T, T] + c[T, T] * sgn[:, None])
    sb = 0.5 * (p.self_blocks + p.self_blocks.transpose(0, 2, 1))
    Z = oracle.fill(p.pos, F, c, sb)
    assert oracle.relerr(Z.T, Z) < 1e-13


def test_far_field_fold():
    """Eq. 1 with d = 1/r is a q = 1 term: Z(c, g) = Z(c + fold(g), 0) with
    fold(g)_{p,1} = -j omega (mu0 / 4 pi) g_p, mu0 / 4 pi = 1e-7 H/m."""
    Nm, P, Q = 2, 3, 2
    p = synth.small(7, Nm, P=P, Q=Q)
    g = synth.complex_normal(np.random.default_rng(3), (Nm, Nm, 2 * P + 1)) * 50.0
    Zg = oracle.fill(p.pos, F, p.coef, p.self_blocks, ff=g)
    c2 = p.coef.copy()
    c2[:, :, :, 1] += -1j * 2 * math.pi * F * 1e-7 * g
    Zf = oracle.fill(p.pos, F, c2, p.self_blocks)
    assert oracle.relerr(Zg, Zf) < 1e-14
    # and the term is really there
    assert oracle.relerr(Zg, oracle.fill(p.pos, F, p.coef, p.self_blocks)) > 1e-3


def test_far_field_alone_matches_eq1():
    """c = 0 and one isotropic pattern product g_0 = 1: Z_app is
    -j omega mu0 e^{-jkr} / (4 pi r) (Eq. 1)."""
    pos = np.array([[0.0, 0.0], [1.7, 2.2]])
    c = _coef_zero(1, 0, 0)
    g = np.ones((1, 1, 1), dtype=np.complex128)
    Z = oracle.fill(pos, F, c, np.zeros((2, 1, 1), np.complex128), ff=g)
    r = math.hypot(1.7, 2.2)
    mu0 = 4e-7 * math.pi
    expect = -1j * (2 * math.pi * F) * mu0 * np.exp(-1j * K * r) / (4 * math.pi * r)
    assert Z[1, 0] == pytest.approx(expect, rel=1e-14)
    assert Z[0, 1] == pytest.approx(expect, rel=1e-14)


def test_coincident_antennas_rejected():
    pos = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 0.0]])
    c = synth.harp_coefficients(1, 1, 1, 1)
    with pytest.raises(ValueError):
        oracle.fill(pos, F, c, np.ones((3, 1, 1), np.complex128))


def test_index_mapping_block_layout():
    """Row m*Nm+T / column n*Nm+S carries testing MBF T of antenna m and
    source MBF S of antenna n: a coefficient table that is nonzero for one
    (T, S) only lights exactly those entries of every mutual block."""
    Nm = 3
    p = synth.small(5, Nm, P=1, Q=1)
    c = _coef_zero(Nm, 1, 1)
    c[2, 0, 1, 0] = 1.0  # T = 2, S = 0, p = 0, q = 0
    Z = oracle.fill(p.pos, F, c, np.zeros((5, Nm, Nm), np.complex128))
    nz = np.argwhere(Z != 0)
    assert len(nz) == 5 * 4
    for i, j in nz:
        assert i % Nm == 2 and j % Nm == 0 and i // Nm != j // Nm


def test_layout_generator_respects_disc_and_separation():
    pos = synth.disc_layout(256, 19.0, 1.5, 2000)
    assert pos.shape == (256, 2)
    assert np.all(np.hypot(pos[:, 0], pos[:, 1]) <= 19.0)
    d = np.hypot(pos[:, None, 0] - pos[None, :, 0], pos[:, None, 1] - pos[None, :, 1])
    d[np.arange(256), np.arange(256)] = np.inf
    assert d.min() >= 1.5
    assert np.array_equal(pos, synth.disc_layout(256, 19.0, 1.5, 2000))


def test_physical_set_removes_exactly_the_q0_part():
    """The fill is linear in c, so Z(c) - Z(c with c_p0 = 0) is the q = 0
    part alone: e^{-jkr} sum_p c_p0 e^{j p alpha} (Eq. 3, 4) in every mutual
    block, zero in the self blocks. Without it each mutual entry is bounded
    by sum_{p, q >= 1} |c_pq| d^q, which decays with distance."""
    p = synth.small(12, 3, P=2, Q=3)
    ph = synth.physical(p)
    assert np.all(ph.coef[..., 0] == 0) and np.array_equal(ph.coef[..., 1:], p.coef[..., 1:])
    assert ph.pos is p.pos and ph.self_blocks is p.self_blocks
    Z = _blocks(oracle.fill(p.pos, F, p.coef, p.self_blocks), p.Na, p.Nm)
    Zp = _blocks(oracle.fill(ph.pos, F, ph.coef, ph.self_blocks), p.Na, p.Nm)
    harm = np.arange(-p.P, p.P + 1)
    for m, n in _pairs(p.Na):
        dx, dy = p.pos[m] - p.pos[n]
        r, alpha = math.hypot(dx, dy), math.atan2(dy, dx)
        q0 = np.exp(-1j * K * r) * np.einsum("tsp,p->ts", p.coef[..., 0],
                                              np.exp(1j * harm * alpha))
        np.testing.assert_allclose(Z[m, n] - Zp[m, n], q0, rtol=0, atol=1e-13 * np.abs(q0).max())
        bound = np.einsum("tspq,q->ts", np.abs(p.coef[..., 1:]), r ** -np.arange(1.0, p.Q + 1))
        assert np.all(np.abs(Zp[m, n]) <= bound * (1 + 1e-12))
    for a in range(p.Na):
        assert np.array_equal(Zp[a, a], p.self_blocks[a])
