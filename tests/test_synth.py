"""Input generator checks that need no GPU."""
import numpy as np

from paper_1702_03781_gb300 import synth


def test_wideband_plan():
    """64 frequencies over 50-350 MHz, MBF count rising linearly 6..20."""
    plan = synth.wideband_plan(64)
    assert plan[0] == (50e6, 6) and plan[-1] == (350e6, 20)
    assert all(6 <= nm <= 20 for _, nm in plan)
    assert [nm for _, nm in plan] == sorted(nm for _, nm in plan)


def test_problem_shapes():
    p = synth.station()
    assert (p.Na, p.Nm, p.N, p.K) == (256, 12, 3072, 102)
    assert p.coef.shape == (12, 12, 17, 6)
    assert p.self_blocks.shape == (256, 12, 12)
    assert p.V.shape == (3072, 256)
    t = synth.tiny()
    assert (t.Na, t.Nm, t.N, t.K) == (16, 4, 64, 36)


def test_self_blocks_follow_the_recipe():
    """Reading 10: A ~ CN(0, 1) from the block seed, then the real margin
    sum_{S != T} |A_TS| + 1 added to each diagonal entry. That boosts the
    diagonal well above its row (|A_TT| >= off-diagonal sum + 1 - |a_TT|)
    without making every row strictly dominant."""
    import numpy as np
    raw = synth.complex_normal(np.random.default_rng(7), (32, 5, 5))
    off = np.abs(raw).sum(axis=2) - np.abs(np.diagonal(raw, axis1=1, axis2=2))
    expect = raw.copy()
    expect[:, np.arange(5), np.arange(5)] += off + 1.0
    sb = synth.self_blocks(32, 5, seed=7)
    assert np.array_equal(sb, expect)
    diag = np.abs(np.diagonal(sb, axis1=1, axis2=2))
    rows = np.abs(sb).sum(axis=2) - diag
    raw_diag = np.abs(np.diagonal(raw, axis1=1, axis2=2))
    assert np.all(diag >= rows + 1.0 - raw_diag - 1e-12)


def test_coefficients_scale_as_two_to_minus_q():
    """c_pq ~ CN(0, 1) 2^-q (reading 3): E|c_pq|^2 = 4^-q for every power q."""
    import numpy as np
    c = synth.harp_coefficients(12, 8, 5, seed=3)
    m2 = (np.abs(c) ** 2).mean(axis=(0, 1, 2))  # 12 * 12 * 17 = 2448 samples per q
    np.testing.assert_allclose(m2 * 4.0 ** np.arange(6), 1.0, rtol=0.1)


def test_seed_plan_is_deterministic_and_distinct():
    """Seeds 1000 c + layout, 1000 c + 100 + i (coefficients), 1000 c + 200 + i
    (self blocks): the same problem twice is identical; different
    frequencies draw different coefficients on the same layout."""
    import numpy as np
    a, b = synth.station(), synth.station()
    assert np.array_equal(a.pos, b.pos) and np.array_equal(a.coef, b.coef)
    assert np.array_equal(a.self_blocks, b.self_blocks)
    w = synth.wideband(3)
    assert all(np.array_equal(w[0].pos, q.pos) for q in w)
    assert not np.array_equal(w[0].self_blocks[:, :6, :6], w[1].self_blocks[:, :6, :6])
    assert np.array_equal(w[0].pos, synth.station().pos)  # the station layout


def test_port_rhs_selects_mbf0_of_each_antenna():
    import numpy as np
    V = synth.port_rhs(5, 3)
    assert V.shape == (15, 5) and V.dtype == np.complex128
    assert np.array_equal(np.argwhere(V == 1.0), np.array([[0, 0], [3, 1], [6, 2], [9, 3],
                                                          [12, 4]]))
    assert np.count_nonzero(V) == 5


def test_large_layout_seeds():
    """The synthesis batch's 8 layouts (1..8) draw distinct seeded positions."""
    p = synth.large(3)
    assert p.meta["layout"] == 3 and (p.Na, p.Nm, p.N) == (1024, 16, 16384)
    pos = [synth.large(layout).pos for layout in range(1, 9)]
    for i in range(8):
        for j in range(i):
            assert not np.array_equal(pos[i], pos[j])
