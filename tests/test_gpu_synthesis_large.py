"""The synthesis batch at full size: 8 seeded random layouts of 1024
antennas x 16 MBFs at 110 MHz (N = 16384, 1024 ports; layout seeds
5001..5008), J and dJ/dpos of each through the library (forward fill and
mixed solve, transposed solve with the cached factors, adjoint kernel).

The oracle's J at this size takes minutes per evaluation (a 16384 x 16384
complex LU), so the full size is checked by properties that hold at any
size; the oracle pins the same code path at the station size
(test_gpu_synthesis.py):
  * every forward and adjoint solve meets the LAPACK tolerance
    sqrt(N) 2^-53 (status 0);
  * translation invariance: Z depends on positions only through differences
    (Eq. 3, 4), so J does too and the gradient sums to zero over the
    antennas, in x and in y;
  * for layout 5001, the directional derivative along a seeded unit
    direction against the Richardson combination of central differences of
    the library's own J (h = 1e-3 m and h/2), within 1e-5 relative. The
    step balances two errors: the plain central difference's O(h^2)
    truncation (4.5e-6 at h = 1e-4 m on the station, so ~5e-4 here before
    Richardson removes it) and the mixed J's rounding noise (relative
    forward error of X, amplified by 1/h).
"""
import numpy as np
import pytest
import torch

from paper_1702_03781_gb300 import synth

pytestmark = pytest.mark.gpu

LAYOUTS = range(1, 9)  # seeds 5001..5008


@pytest.fixture(scope="module")
def harp():
    from paper_1702_03781_gb300 import build
    build.build()
    from paper_1702_03781_gb300.harp import Harp
    h = Harp(0, max_N=16384, max_nrhs=1024)
    yield h
    h.close()


@pytest.fixture(scope="module")
def batch(harp):
    from paper_1702_03781_gb300.synthesis import layout_gradients
    probs = [synth.large(layout) for layout in LAYOUTS]
    return probs, layout_gradients(harp, probs, prec="mixed", max_iter=60)


def test_all_layouts_converge(batch):
    probs, res = batch
    tol = np.sqrt(16384) * 2.0 ** -53
    for p, (J, g, info) in zip(probs, res):
        for leg in ("forward", "adjoint"):
            assert info[leg]["status"] == 0, (p.meta["layout"], leg)
            assert info[leg]["resid"] <= tol, (p.meta["layout"], leg, info[leg])
        assert np.isfinite(J) and J > 0
        assert torch.isfinite(g).all()


def test_translation_invariance(batch):
    _, res = batch
    for J, g, _ in res:
        s = g.sum(dim=0).abs()
        scale = g.abs().sum(dim=0)
        assert torch.all(s <= 1e-9 * scale), (s, scale)


def test_directional_derivative_vs_richardson(harp, batch):
    from paper_1702_03781_gb300.synthesis import port_objective
    probs, res = batch
    p, (J0, g, _) = probs[0], res[0]
    d = "cuda:0"
    coef = torch.from_numpy(p.coef).to(d)
    sb = torch.from_numpy(p.self_blocks).to(d)
    u = np.random.default_rng(5101).standard_normal(p.pos.shape)
    u /= np.linalg.norm(u)

    def J_at(x):
        return float(port_objective(torch.from_numpy(x).to(d), harp, p.freq_hz, coef, sb,
                                    prec="mixed", max_iter=60))

    assert J_at(p.pos) == pytest.approx(J0, rel=1e-12)
    h = 1e-3
    d1 = (J_at(p.pos + h * u) - J_at(p.pos - h * u)) / (2 * h)
    d2 = (J_at(p.pos + h / 2 * u) - J_at(p.pos - h / 2 * u)) / h
    richardson = (4 * d2 - d1) / 3
    gu = float((g.cpu().numpy() * u).sum())
    assert abs(gu - richardson) / abs(richardson) <= 1e-5, (gu, richardson, d1, d2)
