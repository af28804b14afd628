"""Input generator checks that need no GPU."""
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
