"""The benchmark's host-side contract on the CPU: the reference arm's JSON line
(the oracle timed on the host cores), silence on ranks other than 0, and the
clock-record parsing. The GPU arm itself runs only on a GB300."""
import argparse
import io
import json
import os
import sys
from contextlib import redirect_stdout

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_1702_03781_gb300 import synth  # noqa: E402


@pytest.fixture
def tiny_station(monkeypatch):
    # the reference arm's workload, shrunk so the test takes a moment
    monkeypatch.setattr(synth, "station", lambda *a, **k: synth.tiny())
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)


def _run_reference(steps=2, warmup=3):
    args = argparse.Namespace(gpus=1, steps=steps, warmup=warmup, impl="reference")
    buf = io.StringIO()
    with redirect_stdout(buf):
        rc = bench.run_reference(args)
    return rc, buf.getvalue()


def test_reference_arm_prints_one_contract_line(tiny_station):
    rc, out = _run_reference()
    assert rc == 0
    lines = [ln for ln in out.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC
    assert d["unit"] == "ms" and d["higher_is_better"] is False
    assert d["value"] > 0 and d["ms_per_step"] == d["value"]
    assert d["steps"] == 2 and d["warmup"] == 3 and d["n_gpus"] == 1
    assert d["vs_baseline"] is None and d["data"] == "synthetic"
    assert d["config"]["workload"] == bench.WORKLOAD
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1
    assert d["e2e"] == {"value": d["value"], "unit": "ms", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}


def test_reference_arm_is_silent_on_other_ranks(tiny_station, monkeypatch):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    rc, out = _run_reference()
    assert rc == 0 and out == ""


def test_clock_record_parsing():
    lines = ["0, 2070, 2070, 900.5, 0x0, Not Active, Not Active, Not Active, Not Active\n",
             "0, 2055, 2070, 1350.2, 0x4, Not Active, Not Active, Not Active, Active\n",
             "0, 2070, 2070, 1399.0, 0x4, Not Active, Not Active, Not Active, Active\n",
             "garbage\n"]
    s = bench.ClockSampler._parse(lines)
    assert s == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"],
                 "samples": 3}
    slow = bench.ClockSampler._parse(
        ["0, 1500, 2070, 800, 0x8, Active, Not Active, Active, Not Active\n"])
    assert slow["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]
    assert bench.ClockSampler(0).summary()["reasons"] == ["unsampled"]


@pytest.mark.parametrize("K,want", [(102, (8, 9, 36)), (144, (8, 9, 36)), (256, (8, 9, 36)),
                                    (1024, (8, 9, 36)), (4096, (7, 10, 45)), (16384, (6, 12, 66))])
def test_digit_plan_rule(K, want):
    """The bench's restatement of the digit rule that sizes its digit-product
    rooflines: 8-bit digits while K 2^(2b-2) <= 2^24 (one exact FP32 sum),
    then the smallest group count G with b (G - 1) >= 53 + log2(sqrt K) +
    log2 G, and G (G - 1) / 2 digit pairs; values worked out by hand (K = 102:
    8 (G - 1) >= 53 + 3.34 + log2 G first holds at G = 9, 64 >= 59.5)."""
    assert bench._digit_plan(K) == want
