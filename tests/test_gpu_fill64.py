"""GPU parity of the FP64-accurate background fill formed by exact digit
products on the tensor cores (option 'fill64' = 1), through the C ABI,
against the FP64 CPU oracle's fill (Eq. 3 in Eq. 4) and against the
float-float kernel (option 'fill64' = 0).

Tolerances (stated here, derived from the arithmetic):
  * every entry of Z64 within 1e-13 of the largest |Z| entry, and every
    sampled antenna-pair block within 1e-13 of that block's largest entry.
    The digit scheme keeps 9 groups of 8-bit digits of each coefficient row
    and each basis column (scaled by their largest power of two), so its
    dropped terms are below 2^-55 sqrt(K) of max|c| max|phi| per entry
    (about 1e-15 of a block's largest entry here); the oracle's own FP64 sum
    carries K u of the same scale. 1e-13 leaves two orders of margin while a
    wrong digit, group weight or exponent is off by 2^-8 or more.
  * refined solutions: relative Frobenius error <= 1e-10 against the
    solution of the same system filled by the float-float kernel.
Shapes: ragged row tiles (Nm^2 not a multiple of 128), several pair chunks
with a ragged last one (Na^2 above 2048), the station (256 antennas x 12 MBFs,
K = 102) and its variant without the q = 0 terms (every block decays like
1/r, the largest basis value then meets zero coefficients), coincident
antennas, and models outside the kernels' limits (K > 128), which fall back
to the float-float kernel.
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


def _dev(p):
    d = "cuda:0"
    return (torch.from_numpy(p.pos).to(d), torch.from_numpy(p.coef).to(d),
            torch.from_numpy(p.self_blocks).to(d))


def _np(t):
    return t.detach().cpu().numpy()


def _z64(h, p, mode):
    h.set_knob("fill64", mode)
    try:
        pos, coef, sb = _dev(p)
        h.fill(pos, p.freq_hz, coef, sb, prec="mixed")
        return h.z64(p.N).cpu().numpy()
    finally:
        h.set_knob("fill64", 2)


def _check_blocks(Z, Zo, Nm, Na, rng, n=16):
    pairs = [tuple(int(x) for x in rng.choice(Na, 2, replace=False)) for _ in range(n)] if Na > 1 else []
    for m, k in pairs:
        got = Z[m * Nm:(m + 1) * Nm, k * Nm:(k + 1) * Nm]
        want = Zo[m * Nm:(m + 1) * Nm, k * Nm:(k + 1) * Nm]
        assert np.max(np.abs(got - want)) <= 1e-13 * np.max(np.abs(want)), (m, k)


def test_fill64_option_round_trip(harp):
    from paper_1702_03781_gb300.harp import HarpError
    assert harp.knob("fill64") == 2
    for v in (1, 0, 2):
        harp.set_knob("fill64", v)
        assert harp.knob("fill64") == v
    with pytest.raises(HarpError):
        harp.set_knob("fill64", 3)
    assert harp.knob("fill64") == 2


@pytest.mark.parametrize("Na,Nm,P,Q", [(16, 4, 4, 3), (46, 5, 3, 2), (70, 11, 8, 5),
                                       (12, 13, 2, 1), (2, 3, 0, 0), (1, 5, 2, 2),
                                       (33, 1, 1, 4)])
def test_fill64_matches_oracle(harp, Na, Nm, P, Q):
    p = synth.small(Na, Nm, P=P, Q=Q, seed_cfg=61)
    Zo = oracle.fill(p.pos, p.freq_hz, p.coef, p.self_blocks)
    Z = _z64(harp, p, 1)
    assert np.max(np.abs(Z - Zo)) <= 1e-13 * np.max(np.abs(Zo))
    _check_blocks(Z, Zo, Nm, Na, np.random.default_rng(Na * 100 + Nm))
    # the self blocks are copied exactly
    for m in range(min(Na, 4)):
        assert np.array_equal(Z[m * Nm:(m + 1) * Nm, m * Nm:(m + 1) * Nm], p.self_blocks[m])


@pytest.mark.parametrize("physical", [False, True])
def test_fill64_station_matches_oracle_and_float_float(harp, physical):
    p = synth.station()
    if physical:
        p = synth.physical(p)
    Zo = oracle.fill(p.pos, p.freq_hz, p.coef, p.self_blocks)
    Z1 = _z64(harp, p, 1)
    assert np.max(np.abs(Z1 - Zo)) <= 1e-13 * np.max(np.abs(Zo))
    rng = np.random.default_rng(7)
    _check_blocks(Z1, Zo, p.Nm, p.Na, rng, n=32)
    # the farthest pair: its block is the smallest against max|c| max|phi|
    D = np.linalg.norm(p.pos[:, None] - p.pos[None], axis=-1)
    m, k = np.unravel_index(np.argmax(D), D.shape)
    Nm = p.Nm
    blk = (slice(m * Nm, (m + 1) * Nm), slice(k * Nm, (k + 1) * Nm))
    assert np.max(np.abs(Z1[blk] - Zo[blk])) <= 1e-13 * np.max(np.abs(Zo[blk]))
    Z0 = _z64(harp, p, 0)
    assert np.max(np.abs(Z1 - Z0)) <= 1e-13 * np.max(np.abs(Zo))


@pytest.mark.parametrize("P,Q", [(10, 6), (1, 33)])
def test_fill64_outside_the_kernel_limits_falls_back(harp, P, Q):
    # K = 21 x 7 = 147 > 128, or Q > 31: the float-float kernel serves
    p = synth.small(20, 3, P=P, Q=Q, seed_cfg=62)
    Zo = oracle.fill(p.pos, p.freq_hz, p.coef, p.self_blocks)
    Z = _z64(harp, p, 1)
    assert np.max(np.abs(Z - Zo)) <= 1e-13 * np.max(np.abs(Zo))


def test_fill64_coincident_antennas(harp):
    from paper_1702_03781_gb300.harp import HarpError
    p = synth.small(24, 3, P=3, Q=2, seed_cfg=63)
    p.pos[5] = p.pos[17]
    Zs = {}
    for mode in (1, 0):
        harp.set_knob("fill64", mode)
        try:
            pos, coef, sb = _dev(p)
            harp.fill(pos, p.freq_hz, coef, sb, prec="mixed")
            with pytest.raises(HarpError):
                harp.sync()
            Zs[mode] = harp.z64(p.N).cpu().numpy()
        finally:
            harp.set_knob("fill64", 2)
    Z, Nm = Zs[1], p.Nm
    assert not np.any(Z[5 * Nm:6 * Nm, 17 * Nm:18 * Nm])
    assert not np.any(Z[17 * Nm:18 * Nm, 5 * Nm:6 * Nm])
    assert np.max(np.abs(Z - Zs[0])) <= 1e-13 * np.max(np.abs(Zs[0]))
    # the oracle refuses coincident antennas: the other antennas' blocks
    # against its fill of the array without antenna 17
    keep = [a for a in range(p.Na) if a != 17]
    Zo = oracle.fill(p.pos[keep], p.freq_hz, p.coef, p.self_blocks[keep])
    rows = np.concatenate([np.arange(a * Nm, (a + 1) * Nm) for a in keep])
    Zk = Z[np.ix_(rows, rows)]
    assert np.max(np.abs(Zk - Zo)) <= 1e-13 * np.max(np.abs(Zo))


def test_fill64_station_solve(harp):
    p = synth.station()
    pos, coef, sb = _dev(p)
    out = {}
    for mode in (0, 1):
        harp.set_knob("fill64", mode)
        try:
            Z = harp.fill(pos, p.freq_hz, coef, sb, prec="mixed")
            X, info = harp.solve(Z, None, nrhs=p.Na, prec="mixed", max_iter=10)
            assert info["status"] == 0
            out[mode] = _np(X)
        finally:
            harp.set_knob("fill64", 2)
    rel = np.linalg.norm(out[1] - out[0]) / np.linalg.norm(out[0])
    assert rel <= 1e-10
