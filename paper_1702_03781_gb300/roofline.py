"""Roofline bookkeeping for the benchmark: per-kernel-class device time from
the library's instrumentation (CUDA events around each launch, on the
launching stream) and the peak each class is bounded by.

Peaks:
  * HBM and dense BF16 tensor throughput: MEASURED_PEAKS.json (measured on
    the GB300s this runs on). TF32 tensor peak = measured BF16 peak x the
    nominal TF32/BF16 ratio (1.1 / 2.25 PFLOP/s). The exact-slice residual
    counts the bf16 digit products it executes (8 flops per complex
    multiply-add per digit pair) against the BF16 peak.
  * FP32 and FP64 FMA pipes ("alu"): unit count x SMs x maximum SM clock,
    with the per-SM FMA rates measured by an FMA-loop probe on a GB300
    (FP32 74.9 TFLOP/s, FP64 1.20 TFLOP/s at 1995 MHz): 128 FP32 and 2 FP64
    FMA per clock per SM, 152 SMs, 2070 MHz.
"""
from __future__ import annotations

import ctypes as ct
import hashlib
import json
import os

KINDS = ["fill", "gemm", "residual", "panel", "trsm", "swap", "adjoint", "other", "resid_update",
         "fill_ff"]
N_KINDS = 10
SMS = 152
SM_MAX_MHZ = 2070.0
FP32_PEAK_TFLOPS = 2 * 128 * SMS * SM_MAX_MHZ * 1e6 / 1e12   # 80.55
FP64_PEAK_TFLOPS = 2 * 2 * SMS * SM_MAX_MHZ * 1e6 / 1e12     # 1.259
# Float-float kernels (FP64-accurate on the FP32 pipe): one complex
# multiply-add is 96 FP32 instructions (4 compensated real products of 24
# instructions) for 8 algorithmic flops; the pipe issues 128 instructions per
# clock per SM.
FF_INSTR_PER_CMAC = 96
FF_PEAK_TFLOPS = 128 * SMS * SM_MAX_MHZ * 1e6 * 8 / FF_INSTR_PER_CMAC / 1e12   # 3.357
# The FP64-accurate fill factors Eq. 4 by the order of the basis: per
# antenna-pair entry and per p, Q + 1 complex x real products into a
# double-float accumulator (2 x 12 instructions each), a renormalisation (6)
# and one complex product into the three-float accumulator (4 x 24); that is
# 24 + 102 / (Q + 1) instructions per complex multiply-add of the flat sum
# (8 algorithmic flops), 41 at Q = 5.
FILL_FF_Q = 5
FILL_FF_INSTR_PER_CMAC = 24 + 102 / (FILL_FF_Q + 1)
FILL_FF_PEAK_TFLOPS = 128 * SMS * SM_MAX_MHZ * 1e6 * 8 / FILL_FF_INSTR_PER_CMAC / 1e12  # 7.86
# Double-float (Dot2) residual updates: 4 compensated real products of 12
# instructions, 48 per complex multiply-add.
FF2_INSTR_PER_CMAC = 48
FF2_PEAK_TFLOPS = 128 * SMS * SM_MAX_MHZ * 1e6 * 8 / FF2_INSTR_PER_CMAC / 1e12  # 6.714
TF32_OVER_BF16 = 1.1 / 2.25

_ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
TRAFFIC_FILE = os.path.join(_ROOT, "profiles", "traffic.json")


def begin(h, mask: int = (1 << N_KINDS) - 1):
    from . import harp as H
    H._check("harp_profile_begin", H.lib().harp_profile_begin(h.handle, ct.c_uint(mask)))


def end(h):
    from . import harp as H
    ms = (ct.c_double * N_KINDS)()
    fl = (ct.c_double * N_KINDS)()
    n = (ct.c_longlong * N_KINDS)()
    H._check("harp_profile_end", H.lib().harp_profile_end(h.handle, ms, fl, n))
    return {KINDS[k]: {"ms": ms[k], "flops": fl[k], "launches": n[k]} for k in range(N_KINDS)}


def shares(prof: dict) -> dict:
    tot = sum(v["ms"] for v in prof.values()) or 1.0
    return {k: round(v["ms"] / tot, 4) for k, v in prof.items() if v["launches"]}


def source_hash(kind: str) -> str:
    """Hash of the sources a kernel class is built from (traffic validity)."""
    files = {"fill": ["fill.cu", "ff.cuh"], "gemm": ["lu_tc.cu"],
             "residual": ["ozaki.cu", "ozaki.cuh", "resid.cu", "ff.cuh"],
             "panel": ["panel_cluster.cu", "panel_common.cuh", "panel_calu.cu"], "trsm": ["dense.cu"], "swap": ["dense.cu"],
             "adjoint": ["adjoint.cu"], "other": ["dense.cu"],
             "resid_update": ["ozaki.cu", "ozaki.cuh", "resid.cu", "ff.cuh"],
             "fill_ff": ["fill.cu", "ff.cuh"]}.get(kind, [])
    h = hashlib.sha256()
    for f in files:
        p = os.path.join(_ROOT, "paper_1702_03781_gb300", "csrc", f)
        if os.path.exists(p):
            h.update(open(p, "rb").read())
    return h.hexdigest()[:16]


def peak_for(kind: str, impl: str, peaks: dict):
    """(bound, peak, unit, note) for a kernel class."""
    if impl == "tensor_bf16":
        bf16 = peaks.get("bf16_tflops")
        if bf16:
            return "tensor", bf16, "TFLOP/s", "measured bf16 burst (exact-slice digit products)"
        return "tensor", 1900.0, "TFLOP/s", "fallback bf16 1.9 PF (exact-slice digit products)"
    if impl == "tensor_tf32":
        bf16 = peaks.get("bf16_tflops")
        if bf16:
            return "tensor", bf16 * TF32_OVER_BF16, "TFLOP/s", "measured bf16 burst x 1.1/2.25 (TF32)"
        return "tensor", 1900.0 * TF32_OVER_BF16, "TFLOP/s", "fallback bf16 1.9 PF x 1.1/2.25 (TF32)"
    if impl == "fp32":
        note = "FP32 FMA pipe: 128 FMA/clk/SM x 152 SMs x 2070 MHz"
        if kind == "panel":
            note += "; the pivoted panel is latency-bound (one cluster barrier per column)"
        return "alu", FP32_PEAK_TFLOPS, "TFLOP/s", note
    if impl == "ff2":
        return ("alu", FF2_PEAK_TFLOPS, "TFLOP/s",
                "FP32 pipe at 128 instr/clk/SM x 152 SMs x 2070 MHz, 48 instr per complex MAC "
                "(double-float Dot2)")
    if impl == "ff_fill":
        return ("alu", FILL_FF_PEAK_TFLOPS, "TFLOP/s",
                "FP32 pipe at 128 instr/clk/SM x 152 SMs x 2070 MHz, 41 instr per complex MAC of "
                "the flat sum at Q = 5 (factored float-float fill, FP64-accurate); the background "
                "launch holds 4 GPC-sized clusters, 64 of the 152 SMs")
    if impl == "ff":
        return ("alu", FF_PEAK_TFLOPS, "TFLOP/s",
                "FP32 pipe at 128 instr/clk/SM x 152 SMs x 2070 MHz, 96 instr per complex MAC "
                "(float-float, FP64-accurate)")
    return "alu", FP64_PEAK_TFLOPS, "TFLOP/s", "FP64 FMA pipe: 2 FMA/clk/SM x 152 SMs x 2070 MHz"


def entry(kind: str, impl: str, prof_kind: dict, peaks: dict) -> dict:
    bound, peak, unit, note = peak_for(kind, impl, peaks)
    ms = prof_kind["ms"]
    n = max(1, prof_kind["launches"])
    achieved = (prof_kind["flops"] / (ms * 1e-3)) / 1e12 if ms > 0 else 0.0
    traffic = None
    try:
        t = json.load(open(TRAFFIC_FILE)).get(kind)
        if t and t.get("source_sha") == source_hash(kind) and t.get("impl") == impl:
            traffic = t.get("bytes_per_launch")
    except Exception:
        pass
    return {"kernel": kind, "impl": impl, "bound": bound, "achieved": round(achieved, 4),
            "peak": round(peak, 3), "unit": unit, "frac": round(achieved / peak, 4),
            "traffic": traffic, "launches": prof_kind["launches"],
            "avg_launch_ms": round(ms / n, 5), "flops_per_launch": prof_kind["flops"] / n,
            "peak_source": note + (" (of measured)" if bound == "tensor" else
                                   " (derived from unit counts and the maximum clock)")}
