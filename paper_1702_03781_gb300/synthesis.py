"""Differentiable port objective for array synthesis (positions -> J).

J(x) = sum_mn |(E^T Z(x)^{-1} E)_mn|^2, with Z(x) the reduced MBF matrix of
the HARP model (Eq. 3, 4) for antenna positions x. The forward pass fills Z
and solves for the port excitations; the backward pass solves the adjoint
system Z^T Lambda = E conj(P) with the factors cached by the forward solve
and calls the library's adjoint kernel, which recomputes the derivatives of
the fill (Eq. 3, 4 differentiated in r and alpha) instead of storing them.
All arithmetic runs in libharp_gb300.so; this module wires it into autograd.
"""
from __future__ import annotations

import torch

from . import harp as H


class PortObjective(torch.autograd.Function):
    """J = PortObjective.apply(pos, harp, freq_hz, coef, self_blocks, prec,
    max_iter, info).

    `harp` is an H.Harp context; its cached factorisation is used by the
    backward pass, so no other solve may run on it between forward and
    backward. `prec` is "fp64" or "mixed".
    """

    @staticmethod
    def forward(ctx, pos, harp, freq_hz, coef, self_blocks, prec="mixed", max_iter=10,
                info=None):
        Nm = coef.shape[0]
        Na = pos.shape[0]
        Z = harp.fill(pos.detach(), freq_hz, coef, self_blocks,
                      prec="fp64" if prec == "fp64" else "mixed")
        X, fwd = harp.solve(Z, None, nrhs=Na, prec=prec, max_iter=max_iter)
        _, J, W = H.port_objective(X, Na, Nm, want_P=False, want_W=True)
        ctx.harp, ctx.freq_hz, ctx.prec, ctx.max_iter = harp, freq_hz, prec, max_iter
        ctx.save_for_backward(pos.detach(), coef, X, W)
        ctx.info = info if info is not None else {}
        ctx.info["forward"] = fwd
        return J

    @staticmethod
    def backward(ctx, gJ):
        pos, coef, X, W = ctx.saved_tensors
        h = ctx.harp
        # Lambda from the cached factors (FP32 LU with FP64-accurate
        # refinement in the mixed mode)
        Lam, adj = h.solve(None, W, prec=ctx.prec, trans="T", max_iter=ctx.max_iter)
        ctx.info["adjoint"] = adj
        # The contraction G = Lambda X^T with the recomputed derivatives is
        # FP64-accurate: in FP64 on the FP64 path, in double-float on the
        # FP32 pipe on the mixed path (summed over ~Na partners per antenna
        # with cancellation, a plain FP32 contraction leaves ~1e-6 relative
        # error in the gradient at the station size, above the synthesis
        # tolerance).
        grad = h.fill_adjoint(pos, ctx.freq_hz, coef, Lam, X,
                              prec="fp64" if ctx.prec == "fp64" else "mixed")
        return grad * gJ, None, None, None, None, None, None, None


def port_objective(pos, harp, freq_hz, coef, self_blocks, prec="mixed", max_iter=10, info=None):
    """J (0-d float64 tensor); `info`, when given, receives the forward and
    adjoint solves' {'iters', 'resid', 'status'} under "forward" and
    "adjoint" (the latter once backward has run)."""
    return PortObjective.apply(pos, harp, freq_hz, coef, self_blocks, prec, max_iter, info)


def layout_gradients(harp, problems, prec="mixed", max_iter=60):
    """J and dJ/dpos of every problem (one antenna layout each, all of the
    same size), one after another on one context: the synthesis batch.
    Returns [(J float, grad (Na, 2) float64 tensor, info dict)]."""
    out = []
    dev = torch.device("cuda", harp.device)
    for p in problems:
        x = torch.from_numpy(p.pos).to(dev).requires_grad_(True)
        coef = torch.from_numpy(p.coef).to(dev)
        sb = torch.from_numpy(p.self_blocks).to(dev)
        info = {}
        J = port_objective(x, harp, p.freq_hz, coef, sb, prec=prec, max_iter=max_iter, info=info)
        J.backward()
        out.append((float(J.detach()), x.grad, info))
    return out


class PortImpedanceObjective(torch.autograd.Function):
    """J = PortImpedanceObjective.apply(pos, harp, harp_p, freq_hz, coef,
    self_blocks, prec, max_iter): the impedance reading of the synthesis
    objective, J = sum_mn |(P^-1)_mn|^2 with P = E^T Z^-1 E.

    `harp` holds Z's factorisation for the backward pass (as for
    PortObjective); `harp_p` is a second context (max_N >= Na) on which P is
    inverted. The backward pass is PortObjective's with the adjoint
    right-hand side E conj(G), G = -Y^H Y Y^H, Y = P^-1.
    """

    @staticmethod
    def forward(ctx, pos, harp, harp_p, freq_hz, coef, self_blocks, prec="mixed", max_iter=10):
        Nm = coef.shape[0]
        Na = pos.shape[0]
        Z = harp.fill(pos.detach(), freq_hz, coef, self_blocks,
                      prec="fp64" if prec == "fp64" else "mixed")
        X, _ = harp.solve(Z, None, nrhs=Na, prec=prec, max_iter=max_iter)
        P, _, _ = H.port_objective(X, Na, Nm, want_P=True, want_W=False)
        _, J, _, W = H.port_impedance(harp_p, P, Nm)
        ctx.harp, ctx.freq_hz, ctx.prec, ctx.max_iter = harp, freq_hz, prec, max_iter
        ctx.save_for_backward(pos.detach(), coef, X, W)
        return J

    @staticmethod
    def backward(ctx, gJ):
        pos, coef, X, W = ctx.saved_tensors
        h = ctx.harp
        Lam, _ = h.solve(None, W, prec=ctx.prec, trans="T", max_iter=ctx.max_iter)
        grad = h.fill_adjoint(pos, ctx.freq_hz, coef, Lam, X,
                              prec="fp64" if ctx.prec == "fp64" else "mixed")
        return grad * gJ, None, None, None, None, None, None, None


def port_impedance_objective(pos, harp, harp_p, freq_hz, coef, self_blocks, prec="mixed",
                             max_iter=10):
    """J (0-d float64 tensor) of the impedance reading; see
    PortImpedanceObjective."""
    return PortImpedanceObjective.apply(pos, harp, harp_p, freq_hz, coef, self_blocks, prec,
                                        max_iter)
