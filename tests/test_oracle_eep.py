"""Pins of the oracle's embedded element patterns (Section II-C, Eq. 5-6)
and of the pattern error of Eq. 8, against facts that do not come from the
oracle itself: closed forms at broadside, a hand-derived two-element case,
the phase a translation must add, linearity, relabelling, and Eq. 6 (the
array-factor form the paper obtains by swapping the sums) evaluated
independently in numpy.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1702_03781_gb300 import synth

C0 = 299792458.0


def _case(Na=9, Nm=3, nports=4, seed=3):
    p = synth.small(Na, Nm, seed_cfg=seed)
    th, ph, ux, uy = synth.direction_grid(15.0, 40.0)
    F = synth.mbf_patterns(Nm, th, ph, seed + 10)
    X = synth.complex_normal(np.random.default_rng(seed), (Na * Nm, nports))
    return p, ux, uy, F, X


def test_broadside_is_the_plain_sum():
    """u = 0: every phase factor is 1, so E = sum_j F_j sum_i c_ij."""
    p, ux, uy, F, X = _case()
    E = oracle.eep(p.pos, p.freq_hz, X, p.Nm, np.zeros(1), np.zeros(1), F[:, :1])
    csum = X.reshape(p.Na, p.Nm, -1).sum(axis=0)  # [j, m]
    ref = np.einsum("cj,jm->cm", F[:, 0, :], csum)
    np.testing.assert_allclose(E[:, :, 0], ref, rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("frac, factor", [(0.5, -1.0), (0.25, 1j)])
def test_two_elements_by_hand(frac, factor):
    """Two antennas on the x axis, spacing frac * lambda, one MBF, looking
    along +x (theta = 90 deg, phi = 0): E = F (c_0 + c_1 e^{j k D}), and
    e^{j k D} = -1 at lambda/2, j at lambda/4."""
    f = 110e6
    lam = C0 / f
    pos = np.array([[0.0, 0.0], [frac * lam, 0.0]])
    F = np.array([[[2.0 - 1.0j]], [[0.5 + 0.25j]]])  # (2, 1, 1)
    X = np.array([[1.0 + 0.5j], [0.3 - 2.0j]])
    E = oracle.eep(pos, f, X, 1, np.ones(1), np.zeros(1), F)
    for comp in range(2):
        want = F[comp, 0, 0] * (X[0, 0] + factor * X[1, 0])
        assert abs(E[comp, 0, 0] - want) <= 1e-12 * abs(want)


def test_translation_adds_the_phase_of_the_shift():
    p, ux, uy, F, X = _case()
    shift = np.array([3.7, -1.2])
    k = 2 * math.pi * p.freq_hz / C0
    E0 = oracle.eep(p.pos, p.freq_hz, X, p.Nm, ux, uy, F)
    E1 = oracle.eep(p.pos + shift, p.freq_hz, X, p.Nm, ux, uy, F)
    phase = np.exp(1j * k * (ux * shift[0] + uy * shift[1]))
    np.testing.assert_allclose(E1, E0 * phase[None, None, :], rtol=1e-12, atol=1e-12)


def test_linear_in_the_currents_and_invariant_under_relabelling():
    p, ux, uy, F, X = _case()
    Y = synth.complex_normal(np.random.default_rng(9), X.shape)
    a, b = 0.7 - 0.2j, -1.3 + 0.4j
    EX = oracle.eep(p.pos, p.freq_hz, X, p.Nm, ux, uy, F)
    EY = oracle.eep(p.pos, p.freq_hz, Y, p.Nm, ux, uy, F)
    EZ = oracle.eep(p.pos, p.freq_hz, a * X + b * Y, p.Nm, ux, uy, F)
    np.testing.assert_allclose(EZ, a * EX + b * EY, rtol=1e-12, atol=1e-12)
    perm = np.random.default_rng(2).permutation(p.Na)
    rows = (perm[:, None] * p.Nm + np.arange(p.Nm)[None, :]).ravel()
    EP = oracle.eep(p.pos[perm], p.freq_hz, X[rows], p.Nm, ux, uy, F)
    np.testing.assert_allclose(EP, EX, rtol=1e-12, atol=1e-12)


def test_array_factor_form_of_eq6():
    """Eq. 6: sum_j F_j AF_j with AF_j = sum_i c_ij e^{jk u.x_i}, here a
    numpy matrix product of the phase matrix and X's MBF rows."""
    p, ux, uy, F, X = _case(Na=12, Nm=4, nports=5)
    k = 2 * math.pi * p.freq_hz / C0
    A = np.exp(1j * k * (np.outer(ux, p.pos[:, 0]) + np.outer(uy, p.pos[:, 1])))  # (D, Na)
    AF = np.einsum("di,ijm->djm", A, X.reshape(p.Na, p.Nm, -1))
    ref = np.einsum("cdj,djm->cmd", F, AF)
    E = oracle.eep(p.pos, p.freq_hz, X, p.Nm, ux, uy, F)
    np.testing.assert_allclose(E, ref, rtol=1e-11, atol=1e-11)


def test_pattern_error_eq8():
    E = synth.complex_normal(np.random.default_rng(4), (2, 7))
    assert np.all(oracle.pattern_error(E, E, 2.0) == 0.0)
    d = np.zeros_like(E)
    d[0] = 3.0 + 4.0j  # |d_theta| = 5
    d[1] = 1j * 12.0   # |d_phi| = 12
    np.testing.assert_allclose(oracle.pattern_error(E + d, E, 2.0), 6.5 * np.ones(7), rtol=1e-14)
