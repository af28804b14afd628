"""GPU parity of the HARP model construction (Section II-A/B) against the
oracle's DFT + library least squares, on the same samples.

Tolerances: both sides work in FP64; the fit goes through a Vandermonde
matrix in d whose condition number reaches ~1e6-1e8 at Q = 5 on these
grids, so the coefficients agree to 1e-7 of their largest magnitude (exact
recovery: 1e-7 as well, against the coefficients the samples came from),
the residuals to 1e-6 relative.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_1702_03781_gb300 import synth

pytestmark = pytest.mark.gpu

C0 = 299792458.0


def _eval_model(coef, d, alpha):
    P = (coef.shape[2] - 1) // 2
    Q = coef.shape[3] - 1
    E = np.exp(1j * np.outer(alpha, np.arange(-P, P + 1)))
    V = d[:, None] ** np.arange(Q + 1)[None, :]
    return np.einsum("lq,tspq,ap->tsla", V, coef, E)


@pytest.fixture(scope="module")
def lib_built():
    from paper_1702_03781_gb300 import build
    build.build()


def _fit(d, B, P, Q):
    from paper_1702_03781_gb300 import harp as H
    c, rms = H.model_fit(torch.from_numpy(d).cuda(), torch.from_numpy(B).cuda(), P, Q)
    return c.cpu().numpy(), rms.cpu().numpy()


@pytest.mark.parametrize("Nm,P,Q,nd,na", [(12, 8, 5, 24, 32), (3, 4, 3, 12, 16), (1, 0, 0, 1, 1),
                                          (5, 2, 1, 7, 5)])
def test_exact_recovery_matches_oracle(lib_built, Nm, P, Q, nd, na):
    coef = synth.harp_coefficients(Nm, P, Q, seed=91)
    d, alpha = synth.model_grid(n_d=nd, n_alpha=na)
    B = _eval_model(coef, d, alpha)
    c, rms = _fit(d, B, P, Q)
    co, rmso = oracle.model_fit(d, B, P, Q)
    scale = np.max(np.abs(coef))
    assert np.max(np.abs(c - coef)) <= 1e-7 * scale
    assert np.max(np.abs(c - co)) <= 1e-7 * scale
    assert np.max(rms) <= 1e-9 * scale


def test_noisy_samples_least_squares_matches_oracle(lib_built):
    P, Q = 8, 5
    coef = synth.harp_coefficients(6, P, Q, seed=92)
    d, alpha = synth.model_grid(n_d=30, n_alpha=40)
    B = _eval_model(coef, d, alpha)
    B = B + 1e-4 * synth.complex_normal(np.random.default_rng(5), B.shape)
    c, rms = _fit(d, B, P, Q)
    co, rmso = oracle.model_fit(d, B, P, Q)
    assert np.max(np.abs(c - co)) <= 1e-7 * np.max(np.abs(co))
    np.testing.assert_allclose(rms, rmso, rtol=1e-6)


def test_round_trip_through_the_gpu_fill(lib_built):
    """The library's own FP64 fill between a source at the origin and a
    testing antenna at (r cos alpha, r sin alpha), times e^{jkr}, sampled
    on the grid and fitted: the fill's coefficients come back."""
    from paper_1702_03781_gb300.harp import Harp
    Nm, P, Q = 3, 4, 3
    f = 110e6
    k = 2 * math.pi * f / C0
    coef = synth.harp_coefficients(Nm, P, Q, seed=93)
    d, alpha = synth.model_grid(n_d=10, n_alpha=12)
    B = np.zeros((Nm, Nm, d.size, alpha.size), dtype=np.complex128)
    sb = torch.zeros((Nm, Nm), dtype=torch.complex128, device="cuda:0")
    ct = torch.from_numpy(coef).cuda()
    with Harp(0, max_N=2 * Nm, max_nrhs=2) as h:
        for l, dl in enumerate(d):
            r = 1.0 / dl
            for a, al in enumerate(alpha):
                pos = torch.tensor([[r * math.cos(al), r * math.sin(al)], [0.0, 0.0]],
                                   dtype=torch.float64, device="cuda:0")
                Z = h.fill(pos, f, ct, sb, prec="fp64").cpu().numpy()
                B[:, :, l, a] = Z[0:Nm, Nm:2 * Nm] * np.exp(1j * k * r)
    c, _ = _fit(d, B, P, Q)
    assert np.max(np.abs(c - coef)) <= 1e-7 * np.max(np.abs(coef))
