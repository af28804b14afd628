"""Pins of the oracle's radius-of-influence matrix (Section II-D, IV-A):
the kept pairs against a direct distance test and symmetry, the limits
RI -> 0 (self blocks only: Na independent solves) and RI -> infinity (the
full matrix), and the kept blocks equal to the full fill's.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1702_03781_gb300 import synth


@pytest.mark.parametrize("RI", [0.5, 3.0, 7.5])
def test_pairs_are_the_close_ones_and_symmetric(RI):
    p = synth.small(80, 1, seed_cfg=121)
    row_ptr, cols = oracle.ri_pairs(p.pos, RI)
    D = np.hypot(*(p.pos[:, None, :] - p.pos[None, :, :]).transpose(2, 0, 1))
    for m in range(p.Na):
        got = cols[row_ptr[m]:row_ptr[m + 1]].tolist()
        want = [n for n in range(p.Na) if n == m or D[m, n] < RI * (1 - 1e-12)]
        borderline = [n for n in range(p.Na) if abs(D[m, n] - RI) <= 1e-9 * RI]
        assert set(want) <= set(got) <= set(want) | set(borderline)
        assert got == sorted(got) and m in got
        for n in got:
            assert m in cols[row_ptr[n]:row_ptr[n + 1]]


def test_limits_and_kept_blocks():
    p = synth.small(30, 3, P=2, Q=2, seed_cfg=122)
    Zf = oracle.fill(p.pos, p.freq_hz, p.coef, p.self_blocks)
    assert np.array_equal(oracle.ri_fill(p.pos, p.freq_hz, p.coef, p.self_blocks, 1e9), Zf)
    Z0 = oracle.ri_fill(p.pos, p.freq_hz, p.coef, p.self_blocks, 1e-9)
    Nm = p.Nm
    X = oracle.solve(Z0, p.V)
    for m in range(p.Na):  # block diagonal: each antenna alone
        sl = slice(m * Nm, (m + 1) * Nm)
        xm = np.linalg.solve(p.self_blocks[m], p.V[sl, m])
        np.testing.assert_allclose(X[sl, m], xm, rtol=1e-12, atol=1e-14)
    Zr = oracle.ri_fill(p.pos, p.freq_hz, p.coef, p.self_blocks, 4.0)
    row_ptr, cols = oracle.ri_pairs(p.pos, 4.0)
    for m in range(p.Na):
        for n in range(p.Na):
            blk = (slice(m * Nm, (m + 1) * Nm), slice(n * Nm, (n + 1) * Nm))
            if n in cols[row_ptr[m]:row_ptr[m + 1]]:
                assert np.array_equal(Zr[blk], Zf[blk])
            else:
                assert not Zr[blk].any()
