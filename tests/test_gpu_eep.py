"""GPU parity of the embedded element patterns (Section II-C, Eq. 5-6) and
the pattern error (Eq. 8), through the C ABI against the FP64 oracle's
term-by-term double sum.

Tolerance: the library forms the phases with FP64 reduction then FP32
sin/cos (~2e-7 rad), the array factors with three-term TF32 products and
FP32 accumulation over the Na antennas (relative ~sqrt(Na) 2^-24), and the
MBF weighting in FP32 over Nm terms: every output within 1e-5 of the
largest |E| of its case, and the relative Frobenius error below 1e-5.
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
    yield h
    h.close()


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _check(E, Eo):
    assert np.max(np.abs(E - Eo)) <= 1e-5 * np.max(np.abs(Eo))
    assert np.linalg.norm(E - Eo) <= 1e-5 * np.linalg.norm(Eo)


@pytest.mark.parametrize("Na,Nm,nports,dth,dph", [(20, 3, 7, 10.0, 30.0), (37, 5, 1, 7.0, 11.0),
                                                  (9, 2, 3, 45.0, 90.0), (70, 4, 70, 5.0, 5.0)])
def test_eep_matches_oracle(harp, Na, Nm, nports, dth, dph):
    """Random currents on random layouts; grids from 8 to ~1300 directions
    (the product runs on the tensor cores from 64 directions and 64
    MBF x port columns up, on the CUDA cores below)."""
    p = synth.small(Na, Nm, seed_cfg=71)
    th, ph, ux, uy = synth.direction_grid(dth, dph)
    F = synth.mbf_patterns(Nm, th, ph, 72)
    X = synth.complex_normal(np.random.default_rng(Na), (p.N, nports))
    E = harp.eep(_t(p.pos), p.freq_hz, _t(X), Nm, _t(ux), _t(uy), _t(F)).cpu().numpy()
    Eo = oracle.eep(p.pos, p.freq_hz, X, Nm, ux, uy, F)
    _check(E, Eo)


def test_station_eep_full_grid_sampled(harp):
    """The station's 256 port patterns on the 1-degree hemisphere grid (91 x
    360 directions, four chunks of directions), from the mixed solution of
    the port excitations, checked on sampled directions and ports."""
    p = synth.station()
    pos, coef, sb = _t(p.pos), _t(p.coef), _t(p.self_blocks)
    Z = harp.fill(pos, p.freq_hz, coef, sb, prec="mixed")
    X, _ = harp.solve(Z, None, nrhs=p.Na, prec="mixed")
    th, ph, ux, uy = synth.direction_grid(1.0, 1.0)
    F = synth.mbf_patterns(p.Nm, th, ph, 73)
    E = harp.eep(pos, p.freq_hz, X, p.Nm, _t(ux), _t(uy), _t(F)).cpu().numpy()
    assert E.shape == (2, p.Na, th.size)
    rng = np.random.default_rng(74)
    ds = rng.choice(th.size, 96, replace=False)
    ms = rng.choice(p.Na, 6, replace=False)
    Xn = X.cpu().numpy()
    Eo = oracle.eep(p.pos, p.freq_hz, Xn[:, ms], p.Nm, ux[ds], uy[ds], F[:, ds])
    _check(E[:, ms][:, :, ds], Eo)


def test_pattern_error_eq8(harp):
    from paper_1702_03781_gb300 import harp as H
    rng = np.random.default_rng(75)
    E = synth.complex_normal(rng, (2, 5, 301)).astype(np.complex64)
    Er = (E + 1e-3 * synth.complex_normal(rng, E.shape)).astype(np.complex64)
    eps = H.pattern_error(_t(E), _t(Er), 3.5).cpu().numpy()
    ref = oracle.pattern_error(E.astype(np.complex128), Er.astype(np.complex128), 3.5)
    np.testing.assert_allclose(eps, ref, rtol=1e-5)
