"""Pins of the oracle's tessellation (Section II-D, Fig. 3): the hexagon
test against the hexagon's vertices and edges, the tile assignment against
a brute-force nearest-centre search, the partition and nesting of the
lists, and the limit R_ext -> infinity, where every subarray is the whole
array and the tessellated currents are the full solve's.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1702_03781_gb300 import synth

S3 = math.sqrt(3.0)


def test_hexagon_vertices_edges_and_outside():
    R = 2.0
    for ang in range(0, 360, 60):  # vertices (flat top: at 0, 60, ... degrees)
        a = math.radians(ang)
        assert oracle.in_hexagon(R * math.cos(a) * (1 - 1e-12), R * math.sin(a) * (1 - 1e-12), R)
        assert not oracle.in_hexagon(R * math.cos(a) * 1.001, R * math.sin(a) * 1.001, R)
    h = 0.5 * S3 * R  # inradius: the top and bottom edges, and the slanted ones
    assert oracle.in_hexagon(0.0, h, R) and not oracle.in_hexagon(0.0, h * 1.0001, R)
    a = math.radians(30.0)
    assert oracle.in_hexagon(h * math.cos(a) * 0.9999, h * math.sin(a) * 0.9999, R)
    assert not oracle.in_hexagon(h * math.cos(a) * 1.0001, h * math.sin(a) * 1.0001, R)


def test_tile_is_the_nearest_centre_by_brute_force():
    R = 1.7
    rng = np.random.default_rng(1)
    pts = rng.uniform(-20, 20, size=(400, 2))
    cents = {(i, j): oracle.hex_center(i, j, R) for i in range(-12, 13) for j in range(-12, 13)}
    for x, y in pts:
        d2 = {k: (x - cx) ** 2 + (y - cy) ** 2 for k, (cx, cy) in cents.items()}
        best = min(d2.values())
        want = min(k for k, v in d2.items() if v == best)
        assert oracle.hex_tile(x, y, R) == want
        # and the nearest centre's hexagon of circumradius R holds the point
        cx, cy = oracle.hex_center(*want, R)
        assert oracle.in_hexagon(x - cx, y - cy, R * (1 + 1e-12))


def test_neighbour_across_the_top_edge():
    R = 3.0
    cx, cy = oracle.hex_center(2, 1, R)
    h = 0.5 * S3 * R
    assert oracle.hex_tile(cx, cy + 0.99 * h, R) == (2, 1)
    assert oracle.hex_tile(cx, cy + 1.01 * h, R) == (2, 2)


@pytest.mark.parametrize("R_in,R_ext", [(4.0, 4.0), (2.5, 1.0), (6.0, 0.0)])
def test_lists_partition_and_nest(R_in, R_ext):
    p = synth.small(150, 2, seed_cfg=101)
    tiles, inner, outer = oracle.tessellate(p.pos, R_in, R_ext)
    assert tiles == sorted(tiles)
    flat = sorted(a for lst in inner for a in lst)
    assert flat == list(range(p.Na))  # every antenna in exactly one inner part
    for lst_in, lst_out in zip(inner, outer):
        assert lst_in == sorted(lst_in) and lst_out == sorted(lst_out)
        assert set(lst_in) <= set(lst_out)
        if R_ext == 0.0:
            # the extended hexagon is the inner one (edges shared with neighbours)
            assert len(lst_out) <= len(lst_in) + 6


def test_infinite_extension_is_the_full_solve():
    p = synth.small(40, 3, P=2, Q=2, seed_cfg=102)
    tiles, inner, outer = oracle.tessellate(p.pos, 3.0, 1e6)
    assert len(tiles) > 1 and all(lst == list(range(p.Na)) for lst in outer)
    X = oracle.solve_tessellated(p.pos, p.freq_hz, p.coef, p.self_blocks, 3.0, 1e6)
    Zo = oracle.fill(p.pos, p.freq_hz, p.coef, p.self_blocks)
    Xf = oracle.solve(Zo, p.V)
    assert np.linalg.norm(X - Xf) <= 1e-12 * np.linalg.norm(Xf)


def test_finite_extension_keeps_currents_on_the_subarray():
    p = synth.small(60, 2, P=2, Q=1, seed_cfg=103)
    R_in, R_ext = 3.0, 2.0
    tiles, inner, outer = oracle.tessellate(p.pos, R_in, R_ext)
    X = oracle.solve_tessellated(p.pos, p.freq_hz, p.coef, p.self_blocks, R_in, R_ext)
    for t in range(len(tiles)):
        off = sorted(set(range(p.Na)) - set(outer[t]))
        rows = (np.asarray(off, dtype=int)[:, None] * p.Nm + np.arange(p.Nm)[None, :]).ravel()
        for m in inner[t]:
            assert np.all(X[rows, m] == 0)
            assert X[m * p.Nm, m] != 0
