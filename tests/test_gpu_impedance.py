"""GPU parity of the impedance reading of the synthesis objective
(J = sum |(P^-1)_mn|^2 with P = E^T Z^-1 E): the library's inverse of the
port response, J, G = -Y^H Y Y^H and the adjoint right-hand side E conj(G)
against numpy on the same P; then J and dJ/dpos through the library
(forward solve, P's FP64 inverse on a second context, transposed solve with
the cached factors, adjoint kernel) against the oracle's
port_impedance_objective_grad.

Tolerances: the kernel outputs within 1e-12 relative (an FP64 solve and
FP64 products of a well-conditioned 37 x 37 matrix); J within 1e-10 on the
small case and within 2 cond(P) times the measured relative difference of
P at the station (J inherits P's error amplified by P's conditioning); the
gradient within 1e-9 (FP64 path) and 1e-6 (mixed path) relative 2-norm,
the bars of the admittance reading (test_gpu_synthesis.py).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1702_03781_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctxs():
    from paper_1702_03781_gb300 import build
    build.build()
    from paper_1702_03781_gb300.harp import Harp
    h = Harp(0, max_N=3072, max_nrhs=256)
    hp = Harp(0, max_N=256, max_nrhs=256)
    yield h, hp
    hp.close()
    h.close()


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_port_impedance_kernels(ctxs):
    from paper_1702_03781_gb300 import harp as H
    _, hp = ctxs
    Na, Nm = 37, 3
    rng = np.random.default_rng(11)
    P = synth.complex_normal(rng, (Na, Na)) + 8.0 * np.eye(Na)
    Y, J, G, W = H.port_impedance(hp, torch.from_numpy(P).cuda(), Nm)
    Yn = np.linalg.inv(P)
    Gn = -(Yn.conj().T @ Yn @ Yn.conj().T)
    assert _rel(Y.cpu().numpy(), Yn) <= 1e-12
    assert float(J) == pytest.approx(np.sum(np.abs(Yn) ** 2), rel=1e-12)
    Gg = G.cpu().numpy()
    assert _rel(Gg, Gn) <= 1e-12
    E = synth.port_rhs(Na, Nm)
    assert np.array_equal(W.cpu().numpy(), E @ np.conj(Gg))


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-9), ("mixed", 1e-6)])
def test_impedance_gradient_small(ctxs, prec, tol):
    from paper_1702_03781_gb300.synthesis import port_impedance_objective
    h, hp = ctxs
    p = synth.small(30, 4, P=3, Q=2, seed_cfg=43)
    d = "cuda:0"
    x = torch.from_numpy(p.pos).to(d).requires_grad_(True)
    J = port_impedance_objective(x, h, hp, p.freq_hz, torch.from_numpy(p.coef).to(d),
                                 torch.from_numpy(p.self_blocks).to(d), prec=prec)
    J.backward()
    Jo, go = oracle.port_impedance_objective_grad(p.pos, p.freq_hz, p.coef, p.self_blocks)
    assert float(J.detach()) == pytest.approx(Jo, rel=1e-10)
    assert _rel(x.grad.cpu().numpy(), go) <= tol


def test_impedance_gradient_station(ctxs):
    """The station: J = sum |Y|^2 with Y = P^-1 carries P's relative error
    amplified by 2 cond(P) (a first-order bound), so J's bar is that bound
    on the measured difference between the library's P and the oracle's
    (itself within the solution's 1e-10 bar); the gradient keeps the mixed
    path's 1e-6."""
    from paper_1702_03781_gb300 import harp as H
    from paper_1702_03781_gb300.synthesis import port_impedance_objective
    h, hp = ctxs
    p = synth.station()
    d = "cuda:0"
    pos, coef, sb = (torch.from_numpy(a).to(d) for a in (p.pos, p.coef, p.self_blocks))
    Zo = oracle.fill(p.pos, p.freq_hz, p.coef, p.self_blocks)
    Po = oracle.solve(Zo, p.V)[np.arange(p.Na) * p.Nm, :]  # E^T X
    X, _ = h.solve(h.fill(pos, p.freq_hz, coef, sb, prec="mixed"), None, nrhs=p.Na,
                   prec="mixed")
    Pg, _, _ = H.port_objective(X, p.Na, p.Nm, want_W=False)
    dP = _rel(Pg.cpu().numpy(), Po)
    assert dP <= 1e-10
    kappa = float(np.linalg.cond(Po))
    x = pos.clone().requires_grad_(True)
    J = port_impedance_objective(x, h, hp, p.freq_hz, coef, sb, prec="mixed")
    J.backward()
    Jo, go = oracle.port_impedance_objective_grad(p.pos, p.freq_hz, p.coef, p.self_blocks)
    tol = max(1e-10, 2.0 * kappa * dP)
    assert abs(float(J.detach()) - Jo) / Jo <= tol, (kappa, dP)
    assert _rel(x.grad.cpu().numpy(), go) <= 1e-6
