"""The allocation-free adjoint entry point against the regular one.

harp_fill_adjoint_noalloc serves callers that cannot allocate device memory:
its scratch is a fixed device array inside the library. It must give the
gradient of harp_fill_adjoint (same kernels, same summation order), call
after call, although every call reuses the same array. This file is named so
that pytest collects it last.
"""
import ctypes as ct

import numpy as np
import pytest
import torch

from paper_1702_03781_gb300 import synth

pytestmark = pytest.mark.gpu


def _setup(prec):
    from paper_1702_03781_gb300 import build
    build.build()
    from paper_1702_03781_gb300.harp import Harp
    p = synth.small(24, 3, P=2, Q=2, seed_cfg=31)
    d = "cuda:0"
    pos, coef, sb = (torch.from_numpy(x).to(d) for x in (p.pos, p.coef, p.self_blocks))
    h = Harp(0, max_N=p.N, max_nrhs=p.Na)
    zprec = "fp64" if prec == "fp64" else "mixed"
    Z = h.fill(pos, p.freq_hz, coef, sb, prec=zprec)
    X, _ = h.solve(Z, None, nrhs=p.Na, prec=prec)
    Pm = X[0::p.Nm, :].conj()
    W = torch.zeros((p.N, p.Na), dtype=torch.complex128, device=d)
    W[0::p.Nm, :] = Pm
    Lam, _ = h.solve(None, W, prec=prec, trans="T")
    return h, p, pos, coef, Lam, X


@pytest.mark.parametrize("prec,ref_prec", [("fp64", "fp64"), ("mixed", "fp32")])
def test_noalloc_matches_regular_entry_point_twice(prec, ref_prec):
    """The no-alloc entry's FP64 mode is the regular FP64 contraction; its
    other modes are the regular entry's FP32 contraction (the regular mixed
    modes' double-float contraction needs a context)."""
    from paper_1702_03781_gb300 import harp as H
    h, p, pos, coef, Lam, X = _setup(prec)
    ref = h.fill_adjoint(pos, p.freq_hz, coef, Lam, X, prec=ref_prec)
    out1 = H.fill_adjoint_noalloc(pos, p.freq_hz, coef, Lam, X, prec=prec)
    out2 = H.fill_adjoint_noalloc(pos, p.freq_hz, coef, Lam, X, prec=prec)
    torch.cuda.synchronize()
    r = ref.cpu().numpy()
    for out in (out1, out2):
        o = out.cpu().numpy()
        # same kernels and summation order: agreement far inside the 1e-10
        # tolerance the gradient tests use
        assert np.linalg.norm(o - r) / np.linalg.norm(r) <= 1e-12
    h.close()


def test_noalloc_after_a_larger_call_gives_the_same_result():
    """A smaller problem after a larger one still gives the regular entry
    point's gradient. (The pair kernel writes every entry it later reads, so
    the larger call's leftovers in the shared array are never read; the
    clearing at the start of each call is a safeguard this test cannot
    observe.)"""
    from paper_1702_03781_gb300 import harp as H
    h, p, pos, coef, Lam, X = _setup("fp64")
    big = synth.small(40, 2, P=1, Q=1, seed_cfg=32)
    d = "cuda:0"
    bpos = torch.from_numpy(big.pos).to(d)
    bcoef = torch.from_numpy(big.coef).to(d)
    bL = torch.randn(big.N, 5, dtype=torch.complex128, device=d)
    bX = torch.randn(big.N, 5, dtype=torch.complex128, device=d)
    H.fill_adjoint_noalloc(bpos, big.freq_hz, bcoef, bL, bX, prec="fp64")
    ref = h.fill_adjoint(pos, p.freq_hz, coef, Lam, X, prec="fp64")
    out = H.fill_adjoint_noalloc(pos, p.freq_hz, coef, Lam, X, prec="fp64")
    r, o = ref.cpu().numpy(), out.cpu().numpy()
    assert np.linalg.norm(o - r) / np.linalg.norm(r) <= 1e-12
    h.close()


def test_noalloc_refuses_tensors_on_two_devices():
    """pos on the GPU and the output on the host: refused in the binding,
    before a pointer reaches the device-agnostic entry point."""
    from paper_1702_03781_gb300 import harp as H
    p = synth.small(8, 2, P=1, Q=1, seed_cfg=33)
    d = "cuda:0"
    pos, coef = torch.from_numpy(p.pos).to(d), torch.from_numpy(p.coef).to(d)
    X = torch.zeros((p.N, p.Na), dtype=torch.complex128, device=d)
    with pytest.raises(ValueError, match="out must be a CUDA tensor"):
        H.fill_adjoint_noalloc(pos, p.freq_hz, coef, X, X,
                               out=torch.empty((p.Na, 2), dtype=torch.float64))
    with pytest.raises(ValueError, match="X must be a CUDA tensor"):
        H.fill_adjoint_noalloc(pos, p.freq_hz, coef, X, X.cpu())


def test_noalloc_rejects_too_many_antennas():
    from paper_1702_03781_gb300 import harp as H
    L = H.lib()
    Na = H.NOALLOC_MAX_NA + 1
    d = "cuda:0"
    pos = torch.zeros((Na, 2), dtype=torch.float64, device=d)
    coef = torch.zeros((1, 1, 1, 1), dtype=torch.complex128, device=d)
    LX = torch.zeros((Na, 1), dtype=torch.complex128, device=d)
    g = torch.zeros((Na, 2), dtype=torch.float64, device=d)
    st = L.harp_fill_adjoint_noalloc(Na, 1, 0, 0, ct.c_void_p(pos.data_ptr()), 1e8,
                                     ct.c_void_p(coef.data_ptr()), ct.c_void_p(LX.data_ptr()),
                                     ct.c_void_p(LX.data_ptr()), Na, 1, ct.c_void_p(g.data_ptr()),
                                     0, None)
    assert st == H.HARP_E_UNSUPPORTED
