"""The benchmark's roofline bookkeeping (no GPU): the class table matches the
library's instrumentation classes, the arithmetic of `achieved` and `frac`,
the choice of peak, and when stored DRAM traffic is reported."""
import json
import os
import re

import pytest

from paper_1702_03781_gb300 import roofline as R

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_classes_match_the_header():
    src = open(os.path.join(ROOT, "include", "harp_gb300.h")).read()
    defs = {m.group(1).lower(): int(m.group(2))
            for m in re.finditer(r"#define HARP_K_(\w+)\s+(\d+)", src)}
    assert int(re.search(r"#define HARP_PROF_KINDS\s+(\d+)", src).group(1)) == R.N_KINDS
    assert len(R.KINDS) == R.N_KINDS
    for name, idx in defs.items():
        assert R.KINDS[idx] == name, (name, idx)


def test_derived_alu_peaks():
    # 128 FP32 and 2 FP64 FMA per clock per SM, 152 SMs, 2070 MHz
    assert R.FP32_PEAK_TFLOPS == pytest.approx(80.55, abs=0.01)
    assert R.FP64_PEAK_TFLOPS == pytest.approx(1.259, abs=0.001)
    # float-float rates: FP32 instruction rate x 8 flops / instructions per complex MAC
    assert R.FILL_FF_INSTR_PER_CMAC == 41
    assert R.FILL_FF_PEAK_TFLOPS == pytest.approx(R.FP32_PEAK_TFLOPS / 2 * 8 / 41, rel=1e-12)
    assert R.FF_PEAK_TFLOPS == pytest.approx(R.FP32_PEAK_TFLOPS / 2 * 8 / 96, rel=1e-12)


def test_entry_arithmetic_and_measured_peak(monkeypatch, tmp_path):
    monkeypatch.setattr(R, "TRAFFIC_FILE", str(tmp_path / "none.json"))
    prof = {"ms": 2.0, "flops": 4.0e12, "launches": 8}  # 2 TFLOP/s over 2 ms
    e = R.entry("gemm", "tensor_tf32", prof, {"bf16_tflops": 2000.0})
    assert e["achieved"] == pytest.approx(2000.0)  # 4e12 flop / 2e-3 s = 2000 TFLOP/s
    assert e["peak"] == pytest.approx(2000.0 * 1.1 / 2.25, rel=1e-6)
    assert e["frac"] == pytest.approx(2000.0 / (2000.0 * 1.1 / 2.25), rel=1e-3)
    assert e["avg_launch_ms"] == pytest.approx(0.25)
    assert e["flops_per_launch"] == pytest.approx(5.0e11)
    assert e["bound"] == "tensor" and "of measured" in e["peak_source"]
    assert e["traffic"] is None


def test_fallback_peak_without_measurements(monkeypatch, tmp_path):
    monkeypatch.setattr(R, "TRAFFIC_FILE", str(tmp_path / "none.json"))
    e = R.entry("residual", "tensor_bf16", {"ms": 1.0, "flops": 1e9, "launches": 1}, {})
    assert e["peak"] == pytest.approx(1900.0) and "fallback" in e["peak_source"]
    a = R.entry("panel", "fp32", {"ms": 1.0, "flops": 1e9, "launches": 1}, {})
    assert a["bound"] == "alu" and a["peak"] == pytest.approx(R.FP32_PEAK_TFLOPS, rel=1e-3)


def test_traffic_reported_only_for_the_captured_sources(monkeypatch, tmp_path):
    f = tmp_path / "traffic.json"
    monkeypatch.setattr(R, "TRAFFIC_FILE", str(f))
    prof = {"ms": 1.0, "flops": 1e9, "launches": 1}
    good = {"bytes_per_launch": 123, "source_sha": R.source_hash("panel"), "impl": "fp32"}
    f.write_text(json.dumps({"panel": good}))
    assert R.entry("panel", "fp32", prof, {})["traffic"] == 123
    # the kernel changed since the capture, or another implementation ran
    f.write_text(json.dumps({"panel": dict(good, source_sha="0" * 16)}))
    assert R.entry("panel", "fp32", prof, {})["traffic"] is None
    f.write_text(json.dumps({"panel": dict(good, impl="ff")}))
    assert R.entry("panel", "fp32", prof, {})["traffic"] is None


def test_committed_traffic_entries_name_known_classes():
    t = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    for k, v in t.items():
        assert k in R.KINDS
        assert v["bytes_per_launch"] > 0 and len(v["source_sha"]) == 16


def test_shares_sum_to_one():
    prof = {k: {"ms": float(i + 1), "flops": 0.0, "launches": 1} for i, k in enumerate(R.KINDS)}
    prof["adjoint"] = {"ms": 0.0, "flops": 0.0, "launches": 0}  # a class that did not run
    s = R.shares(prof)
    assert "adjoint" not in s
    assert sum(s.values()) == pytest.approx(1.0, abs=1e-3)
    assert s["fill_ff"] == pytest.approx(10.0 / 48.0, abs=1e-4)
