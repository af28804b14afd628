"""Host logic of the autotuner: cache keys, loading, applying cached knobs
(a fake context records what is set), and the coordinate descent's
acceptance rule on a fake timing table. No GPU."""
import json

import pytest

from paper_1702_03781_gb300 import autotune


class FakeCtx:
    def __init__(self):
        self.knobs = {}

    def set_knob(self, name, value):
        assert name in autotune.DEFAULTS
        self.knobs[name] = value


def test_key_names_the_class_and_arch(monkeypatch):
    monkeypatch.setattr(autotune, "arch", lambda: "sm_103")
    assert autotune.key(3072, 12, 102) == "N=3072,Nm=12,K=102,arch=sm_103"


def test_load_missing_or_broken_cache(tmp_path):
    assert autotune.load(str(tmp_path / "none.json")) == {}
    bad = tmp_path / "bad.json"
    bad.write_text("{not json")
    assert autotune.load(str(bad)) == {}


def test_apply_defaults_and_cached(monkeypatch, tmp_path):
    monkeypatch.setattr(autotune, "arch", lambda: "sm_103")
    c = FakeCtx()
    assert autotune.apply(c, 64, 4, 45, cache={}) == autotune.DEFAULTS
    assert c.knobs == autotune.DEFAULTS
    cache = {autotune.key(64, 4, 45): {"knobs": {"panel_rows": 96, "splitk_max": 2}}}
    path = tmp_path / "t.json"
    path.write_text(json.dumps(cache))
    c2 = FakeCtx()
    got = autotune.apply(c2, 64, 4, 45, cache=autotune.load(str(path)))
    assert got == dict(autotune.DEFAULTS, panel_rows=96, splitk_max=2)
    assert c2.knobs == got


def test_search_space_is_within_option_ranges():
    # ranges accepted by harp_ctx_set_option
    assert all(32 <= v <= 384 for v in autotune.SPACE["panel_rows"])
    assert all(v >= 0 for v in autotune.SPACE["fill_chunk"])
    assert all(1 <= v <= 8 for v in autotune.SPACE["splitk_max"])
    for name, v in autotune.DEFAULTS.items():
        assert v in autotune.SPACE[name]


def test_descent_keeps_only_clear_wins(monkeypatch):
    """tune_problem's rule on a fake step time: a knob value is kept only
    when it is faster by more than the margin."""
    saving = {("panel_rows", 128): 1.0, ("fill_chunk", 3): 1.0, ("splitk_max", 4): 0.05}

    class Ctx(FakeCtx):
        def __enter__(self):
            return self

        def __exit__(self, *a):
            return False

    ctx = Ctx()

    def fake_time(h, p, dev, reps):
        return 10.0 - sum(ms for (name, v), ms in saving.items() if h.knobs.get(name) == v)

    class P:
        N, Nm, Na = 64, 4, 16

    monkeypatch.setattr(autotune, "_time_step", fake_time)
    monkeypatch.setattr(autotune.H, "Harp", lambda *a, **k: ctx)
    monkeypatch.setattr(autotune.torch, "device", lambda *a: None)
    res = autotune.tune_problem(P(), reps=1)
    # panel_rows 128 and fill_chunk 3 save 10 % each and are kept;
    # splitk_max 4 saves 0.05 of 8 ms (< 1 %) and is dropped; fill_chunk 6
    # exceeds Nm and is never tried
    assert res["knobs"]["panel_rows"] == 128
    assert res["knobs"]["fill_chunk"] == 3
    assert res["knobs"]["splitk_max"] == 8
    assert res["default_ms"] == 10.0
    assert all(t["knobs"]["fill_chunk"] <= P.Nm for t in res["trials"])
