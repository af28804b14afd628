"""GPU parity of the radius-of-influence matrix (Section II-D, IV-A)
against the oracle: kept pairs bit-exact (the same FP64 test without fused
multiply-add), the kept blocks' values within the fill tolerances (FP64:
1e-13 of the largest entry, self blocks bit-exact; FP32: 1e-5 relative
Frobenius), the solution of the sparse system within 1e-10 of the oracle's,
and RI -> infinity giving the dense path's solution.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1702_03781_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H():
    from paper_1702_03781_gb300 import build
    build.build()
    from paper_1702_03781_gb300 import harp
    return harp


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("RI", [0.0, 2.0, 4.5, 1e9])
def test_pairs_bit_exact(H, RI):
    p = synth.small(120, 1, seed_cfg=121)
    rp, ci = H.ri_pairs(_t(p.pos), RI)
    rpo, cio = oracle.ri_pairs(p.pos, RI)
    assert np.array_equal(rp.cpu().numpy(), rpo) and np.array_equal(ci.cpu().numpy(), cio)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_sparse_fill_and_solve_match_oracle(H, prec):
    p = synth.small(50, 3, P=3, Q=2, seed_cfg=123)
    RI = 4.0
    pos, coef, sb = _t(p.pos), _t(p.coef), _t(p.self_blocks)
    rp, ci = H.ri_pairs(pos, RI)
    v64 = H.ri_fill(pos, p.freq_hz, coef, sb, rp, ci, prec="fp64")
    Zo = oracle.ri_fill(p.pos, p.freq_hz, p.coef, p.self_blocks, RI)
    Z64 = H.bsr_to_dense(rp, ci, v64, p.Na).cpu().numpy()
    assert np.max(np.abs(Z64 - Zo)) <= 1e-13 * np.max(np.abs(Zo))
    Nm = p.Nm
    for m in range(p.Na):  # self blocks copied bit for bit
        sl = slice(m * Nm, (m + 1) * Nm)
        assert np.array_equal(Z64[sl, sl], p.self_blocks[m])
    Xo = oracle.solve(Zo, p.V)
    with H.Harp(0, max_N=p.N, max_nrhs=p.Na) as h:
        if prec == "fp64":
            Z = H.bsr_to_dense(rp, ci, v64, p.Na)
        else:
            v32 = H.ri_fill(pos, p.freq_hz, coef, sb, rp, ci, prec="mixed")
            Z = H.bsr_to_dense(rp, ci, v32, p.Na)
            Zf = Z.cpu().numpy().astype(np.complex128)
            assert np.linalg.norm(Zf - Zo) <= 1e-5 * np.linalg.norm(Zo)
            H.bsr_to_dense(rp, ci, v64, p.Na, out=h.z64(p.N))
        X, info = h.solve(Z, None, nrhs=p.Na, prec=prec, max_iter=10)
    assert np.linalg.norm(X.cpu().numpy() - Xo) <= 1e-10 * np.linalg.norm(Xo)


def test_infinite_radius_is_the_dense_path(H):
    p = synth.small(40, 4, P=2, Q=3, seed_cfg=124)
    pos, coef, sb = _t(p.pos), _t(p.coef), _t(p.self_blocks)
    rp, ci = H.ri_pairs(pos, 1e9)
    assert ci.shape[0] == p.Na * p.Na
    v64 = H.ri_fill(pos, p.freq_hz, coef, sb, rp, ci, prec="fp64")
    with H.Harp(0, max_N=p.N, max_nrhs=p.Na) as h:
        Zs = H.bsr_to_dense(rp, ci, v64, p.Na)
        Zd = h.fill(pos, p.freq_hz, coef, sb, prec="fp64")
        assert torch.max(torch.abs(Zs - Zd)).item() <= 1e-13 * torch.max(torch.abs(Zd)).item()
        Xs, _ = h.solve(Zs, None, nrhs=p.Na, prec="fp64")
        Xd, _ = h.solve(Zd, None, nrhs=p.Na, prec="fp64")
    assert (torch.linalg.norm(Xs - Xd) / torch.linalg.norm(Xd)).item() <= 1e-10
