"""GPU parity of the tessellation approach (Section II-D, Section IV-B)
against the oracle: tiles and lists bit-exact (the membership decisions are
the same FP64 operations, no fused multiply-add), the assembled currents
within 1e-10 (relative Frobenius) of the oracle's subarray solves, and the
limit R_ext -> infinity within 1e-10 of the full solve.
"""
import math

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


def _lists(t):
    ip, ii = t.inner_ptr.cpu().numpy(), t.inner_idx.cpu().numpy()
    op, oi = t.outer_ptr.cpu().numpy(), t.outer_idx.cpu().numpy()
    tiles = [tuple(x) for x in t.tiles.cpu().numpy().tolist()]
    inner = [ii[ip[k]:ip[k + 1]].tolist() for k in range(len(tiles))]
    outer = [oi[op[k]:op[k + 1]].tolist() for k in range(len(tiles))]
    return tiles, inner, outer


@pytest.mark.parametrize("Na,R_in,R_ext", [(150, 4.0, 4.0), (300, 2.5, 1.0), (60, 6.0, 0.0),
                                           (40, 3.0, 1e6)])
def test_lists_bit_exact(H, Na, R_in, R_ext):
    p = synth.small(Na, 1, seed_cfg=111)
    t = H.tessellate(torch.from_numpy(p.pos).cuda(), R_in, R_ext)
    assert _lists(t) == oracle.tessellate(p.pos, R_in, R_ext)


def test_lists_bit_exact_on_tile_edges(H):
    """Antennas on shared edges and vertices of the lattice (ties of the
    nearest-centre rule) and on the extended hexagon's edge."""
    R = 2.0
    pts = []
    for i in range(-2, 3):
        for j in range(-2, 3):
            cx, cy = oracle.hex_center(i, j, R)
            h = 0.5 * oracle.SQRT3 * R
            pts += [(cx, cy), (cx, cy + h), (cx + R, cy), (cx + 0.5 * R, cy + h),
                    (cx + 0.75 * R, cy + 0.5 * h)]
    pos = np.array(pts)
    for R_ext in (0.0, 1.0, 2.0):
        t = H.tessellate(torch.from_numpy(pos).cuda(), R, R_ext)
        assert _lists(t) == oracle.tessellate(pos, R, R_ext)


def _contexts(H, t, Nm, n=3):
    sizes = t.sizes()
    return [H.Harp(0, max_N=max(sizes) * Nm, max_nrhs=max(sizes)) for _ in range(n)]


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_tessellated_currents_match_oracle(H, prec):
    p = synth.small(60, 2, P=2, Q=1, seed_cfg=103)
    R_in, R_ext = 3.0, 2.0
    pos = torch.from_numpy(p.pos).cuda()
    t = H.tessellate(pos, R_in, R_ext)
    assert t.n_tiles > 3
    ctxs = _contexts(H, t, p.Nm)
    X = H.solve_tessellated(ctxs, t, pos, p.freq_hz, torch.from_numpy(p.coef).cuda(),
                            torch.from_numpy(p.self_blocks).cuda(), prec=prec)
    for c in ctxs:
        c.close()
    Xo = oracle.solve_tessellated(p.pos, p.freq_hz, p.coef, p.self_blocks, R_in, R_ext)
    Xg = X.cpu().numpy()
    assert np.linalg.norm(Xg - Xo) <= 1e-10 * np.linalg.norm(Xo)
    assert np.array_equal(Xg == 0, Xo == 0)  # the same zero pattern


def test_infinite_extension_gives_the_full_solve(H):
    p = synth.small(48, 3, P=2, Q=2, seed_cfg=102)
    pos = torch.from_numpy(p.pos).cuda()
    t = H.tessellate(pos, 3.0, 1e6)
    assert t.n_tiles > 1
    ctxs = _contexts(H, t, p.Nm, n=2)
    X = H.solve_tessellated(ctxs, t, pos, p.freq_hz, torch.from_numpy(p.coef).cuda(),
                            torch.from_numpy(p.self_blocks).cuda(), prec="mixed")
    for c in ctxs:
        c.close()
    Zo = oracle.fill(p.pos, p.freq_hz, p.coef, p.self_blocks)
    Xf = oracle.solve(Zo, p.V)
    assert np.linalg.norm(X.cpu().numpy() - Xf) <= 1e-10 * np.linalg.norm(Xf)
