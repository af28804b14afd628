"""Pins of the oracle's HARP model construction (Section II-A/B: DFT over
the angle, least-squares polynomial in d = 1/r): exact recovery of a
band-limited model, the least-squares optimality of the fit on noisy
samples, a single harmonic giving a single DFT line, and the round trip
through the oracle's own fill (samples of Eq. 4 between two antennas,
divided by e^{-jkr}, rebuild the coefficients the fill was given).
"""
import math

import numpy as np
import pytest

import oracle
from paper_1702_03781_gb300 import synth

C0 = 299792458.0


def _eval_model(coef, d, alpha):
    """Eq. 3 at the grid points: B[T, S, l, a]."""
    P = (coef.shape[2] - 1) // 2
    Q = coef.shape[3] - 1
    E = np.exp(1j * np.outer(alpha, np.arange(-P, P + 1)))  # (Na, np)
    V = d[:, None] ** np.arange(Q + 1)[None, :]              # (Nd, nq)
    return np.einsum("lq,tspq,ap->tsla", V, coef, E)


@pytest.mark.parametrize("Nm,P,Q,nd,na", [(3, 4, 3, 12, 16), (2, 8, 5, 24, 17), (1, 0, 0, 1, 1)])
def test_band_limited_model_is_recovered_exactly(Nm, P, Q, nd, na):
    """With n_alpha >= 2P + 1 and n_d >= Q + 1 the samples determine c."""
    coef = synth.harp_coefficients(Nm, P, Q, seed=81)
    d, alpha = synth.model_grid(n_d=nd, n_alpha=na)
    c, rms = oracle.model_fit(d, _eval_model(coef, d, alpha), P, Q)
    assert np.max(np.abs(c - coef)) <= 1e-9 * np.max(np.abs(coef))
    assert np.max(rms) <= 1e-12 * np.max(np.abs(coef))


def test_too_few_angles_alias():
    """n_alpha < 2P + 1: the harmonics p and p - n_alpha share their samples,
    so a model using both cannot be recovered."""
    coef = np.zeros((1, 1, 5, 1), dtype=np.complex128)
    coef[0, 0, 0, 0] = 1.0  # p = -2
    coef[0, 0, 4, 0] = 1.0  # p = +2
    d, alpha = synth.model_grid(n_d=3, n_alpha=4)  # e^{2j a} = e^{-2j a} on 4 angles
    c, _ = oracle.model_fit(d, _eval_model(coef, d, alpha), 2, 0)
    assert np.max(np.abs(c - coef)) > 0.5


def test_least_squares_optimality_on_noisy_samples():
    """Noisy samples: the residual of each harmonic's fit is orthogonal to
    the powers of d (the normal equations of the fit)."""
    P, Q = 3, 4
    coef = synth.harp_coefficients(2, P, Q, seed=82)
    d, alpha = synth.model_grid(n_d=20, n_alpha=16)
    B = _eval_model(coef, d, alpha)
    B = B + 1e-3 * synth.complex_normal(np.random.default_rng(3), B.shape)
    c, rms = oracle.model_fit(d, B, P, Q)
    V = d[:, None] ** np.arange(Q + 1)[None, :]
    W = np.exp(-1j * np.outer(alpha, np.arange(-P, P + 1))) / alpha.size
    for T in range(2):
        for S in range(2):
            b = B[T, S] @ W
            r = b - V @ c[T, S].T
            assert np.max(np.abs(V.T @ r)) <= 1e-10 * np.max(np.abs(V.T @ b))
    assert 0.5e-3 < np.max(rms) < 2e-3


def test_single_harmonic_is_one_dft_line():
    d, alpha = synth.model_grid(n_d=6, n_alpha=12)
    B = np.exp(3j * alpha)[None, None, None, :] * (0.5 + d)[None, None, :, None]
    c, _ = oracle.model_fit(d, B, 5, 1)
    want = np.zeros((1, 1, 11, 2), dtype=np.complex128)
    want[0, 0, 5 + 3] = [0.5, 1.0]
    assert np.max(np.abs(c - want)) <= 1e-12


def test_round_trip_through_the_fill():
    """Samples of the oracle's fill (Eq. 3 in Eq. 4, d = 1/r) for a testing
    antenna at (r cos alpha, r sin alpha) of a source at the origin, times
    e^{jkr}, are B itself: the construction returns the fill's coefficients."""
    Nm, P, Q = 2, 3, 2
    f = 110e6
    k = 2 * math.pi * f / C0
    coef = synth.harp_coefficients(Nm, P, Q, seed=83)
    d, alpha = synth.model_grid(n_d=8, n_alpha=9)
    sb = np.zeros((2, Nm, Nm), dtype=np.complex128)
    B = np.zeros((Nm, Nm, d.size, alpha.size), dtype=np.complex128)
    for l, dl in enumerate(d):
        r = 1.0 / dl
        for a, al in enumerate(alpha):
            pos = np.array([[r * math.cos(al), r * math.sin(al)], [0.0, 0.0]])
            Z = oracle.fill(pos, f, coef, sb)
            B[:, :, l, a] = Z[0:Nm, Nm:2 * Nm] * np.exp(1j * k * r)
    c, _ = oracle.model_fit(d, B, P, Q)
    assert np.max(np.abs(c - coef)) <= 1e-9 * np.max(np.abs(coef))
