"""Benchmark: HARP fill + MBF solve per frequency on the 256-antenna station.

One step = one pass of the hot path for one frequency of the 256-antenna,
12-MBF SKA-like station at 110 MHz (N = 3072 unknowns, 256 port
excitations): the mixed-precision fill (harp_fill) and the mixed-precision
solve with iterative refinement to the FP64 backward-error tolerance
(mbf_solve), all through the library's C ABI. The plain FP64 GPU path is
timed beside it on the same inputs, and both solutions are checked against
each other (and, in the tests, against the FP64 CPU oracle).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Under torchrun each rank runs an independent replica (the solve does not
shard); value = max-over-ranks step time / frequencies processed by all
ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "fill+solve ms/frequency (256 ant, 12 MBF), mixed vs FP64 GPU at ≤1e-10 rel err"
WORKLOAD = "SKA-like station: 256 antennas in a 38 m disc (min sep 1.5 m), 12 MBFs, 110 MHz, P=8, Q=5; N=3072, 256 port RHS"


# Arithmetic each kernel class runs on in the mixed step (roofline bound).
IMPL = {"fill": "fp32", "gemm": "tensor_tf32", "residual": "ff", "panel": "fp32",
        "trsm": "fp32", "swap": "fp32", "adjoint": "fp32", "other": "fp32", "resid_update": "ff2",
        "fill_ff": "ff_fill"}
# Kernel classes that do the step's arithmetic (the others are glue: row
# swaps, triangular leaves, conversions); the residual classes run on the
# bf16 tensor cores when the context uses the exact-slice residual.
COMPUTE_KINDS = ("fill", "fill_ff", "gemm", "residual", "resid_update")


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clock/throttle samples while the timed region runs."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None
        self._summary = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(prefix=f"harp_clocks{self.index}_", suffix=".csv")
            self.f = os.fdopen(fd, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        lines = []
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()
            with open(self.path) as f:
                lines = f.readlines()
        if self.path:
            os.unlink(self.path)
        self._summary = self._parse(lines) if self.proc else None

    @staticmethod
    def _parse(lines):
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in lines:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}

    def summary(self):
        return self._summary or {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}


def wideband_throughput(device: int, n_ctx: int | None = None, n_freq: int = 64) -> dict:
    """Config 3: the station layout at n_freq frequencies over 50-350 MHz
    (Nm 6..20, N 1536..5120, 256 ports each), filled and solved (mixed, to
    the LAPACK tolerance) by the library's batch scheduler. The worker
    count and each context's tile-shape knobs come from the autotuner's
    cache when it holds the wideband batch (else 4 workers, default knobs).
    One warm-up batch of n_ctx frequencies, then one timed batch of all of
    them: device time from CUDA events on every worker's stream (first
    start to last end) and host wall clock around the synchronous call."""
    import torch
    from paper_1702_03781_gb300 import autotune
    from paper_1702_03781_gb300 import harp as H
    from paper_1702_03781_gb300 import synth
    d = f"cuda:{device}"
    cache = autotune.load()
    tuned = cache.get("wideband_batch")
    if n_ctx is None:
        n_ctx = int(tuned["workers"]) if tuned else 4
    probs = synth.wideband(n_freq)
    items = [H.BatchItem(torch.from_numpy(q.pos).to(d), q.freq_hz, torch.from_numpy(q.coef).to(d),
                         torch.from_numpy(q.self_blocks).to(d)) for q in probs]
    max_N = max(it.N for it in items)
    mid = sorted(probs, key=lambda q: q.N)[len(probs) // 2]
    ctxs = [H.Harp(device, max_N=max_N, max_nrhs=256) for _ in range(n_ctx)]
    knobs = [autotune.apply(c, mid.N, mid.Nm, mid.K, cache) for c in ctxs][0]
    for name in ("inverses", "fill64"):
        if tuned and name in tuned:
            for c in ctxs:
                c.set_knob(name, int(tuned[name]))
            knobs = dict(knobs, **{name: int(tuned[name])})
    H.solve_batch(ctxs, items[-n_ctx:], prec="mixed")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    H.solve_batch(ctxs, items, prec="mixed", check=False)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    dev_ms = ctxs[0].batch_device_ms()
    ok = all(it.status == 0 for it in items)
    iters = [it.iters for it in items]
    for c in ctxs:
        c.close()
    return {"frequencies": n_freq, "contexts": n_ctx, "N_range": [min(it.N for it in items), max_N],
            "device_ms_per_frequency": round(dev_ms / n_freq, 3),
            "ms_per_frequency": round(1e3 * wall / n_freq, 3), "wall_ms": round(1e3 * wall, 2),
            "device_ms": round(dev_ms, 2), "all_converged": ok,
            "corrections": [min(iters), max(iters)], "knobs": knobs,
            "tuned": bool(tuned) and autotune.key(mid.N, mid.Nm, mid.K) in cache,
            "timing": "device: CUDA events on every worker stream, first start to last end; "
                      "wall: host clock around one synchronous batch call"}


def method_work(N: int, nrhs: int, K: int, prof: dict, info: dict, peaks: dict,
                fp64_ms: float, mixed_ms: float) -> dict:
    """The step's algorithmic work per part, from the per-class device times
    of one instrumented step:
      * residual: R = V - Z X with Z the FP64 matrix, 8 N^2 nrhs flops and
        16 N^2 + (8 + 16 + 16) N nrhs bytes (Z64, X as FP32 planes, V and R
        in FP64) per residual; the first residual of a solve is one call
        (class 'residual'), each correction adds one update ('resid_update');
      * LU: (8/3) N^3 flops (complex) over the summed device time of the
        factorisation's classes (panel, gemm, trsm, swap; the factor
        inverses and the correction solves run in 'gemm' too, so this
        rate is a lower bound), against the TF32 peak and the three-term
        TF32 effective peak (a third of it);
      * the FP64 GPU path against its bound: fill (8 K N^2) + LU + two
        triangular solves (8 N^2 nrhs) flops at the FP64 FMA peak."""
    from paper_1702_03781_gb300 import roofline
    hbm = peaks.get("hbm_gbs") or 6800.0
    bf16 = peaks.get("bf16_tflops") or 1900.0
    tf32 = bf16 * roofline.TF32_OVER_BF16
    res_flops = 8.0 * N * N * nrhs
    res_bytes = 16.0 * N * N + 40.0 * N * nrhs
    out = {}
    calls = {"residual": 1, "resid_update": int(info.get("iters") or 0)}
    for kind, n in calls.items():
        pk = prof.get(kind, {})
        if not pk.get("launches") or n < 1:
            continue
        ms = pk["ms"] / n
        t = None
        try:
            tj = json.load(open(roofline.TRAFFIC_FILE)).get(kind)
            if tj and tj.get("source_sha") == roofline.source_hash(kind):
                t = tj["bytes_per_launch"] * pk["launches"] / n
        except Exception:
            pass
        out[kind] = {"calls_per_step": n, "ms_per_call": round(ms, 4),
                     "flops_per_call": res_flops, "bytes_per_call": res_bytes,
                     "tflops": round(res_flops / (ms * 1e-3) / 1e12, 3),
                     "gbs": round(res_bytes / (ms * 1e-3) / 1e9, 1),
                     "frac_hbm": round(res_bytes / (ms * 1e-3) / 1e9 / hbm, 4),
                     "digit_product_tflops": round(pk["flops"] / (pk["ms"] * 1e-3) / 1e12, 2),
                     "digit_product_frac_bf16": round(pk["flops"] / (pk["ms"] * 1e-3) / 1e12 / bf16,
                                                      4),
                     "traffic_per_call": t,
                     "traffic_over_algorithmic": round(t / res_bytes, 2) if t else None}
    lu_flops = 8.0 / 3.0 * N ** 3
    lu_ms = sum(prof.get(k, {}).get("ms", 0.0) for k in ("panel", "gemm", "trsm", "swap"))
    if lu_ms > 0:
        ach = lu_flops / (lu_ms * 1e-3) / 1e12
        out["lu"] = {"flops": lu_flops, "device_ms_sum": round(lu_ms, 3),
                     "tflops": round(ach, 3), "frac_tf32": round(ach / tf32, 4),
                     "frac_3xtf32_effective": round(3 * ach / tf32, 4),
                     "peak_tf32": round(tf32, 1),
                     "note": "classes panel+gemm+trsm+swap summed over their launches"}
    fp64_flops = 8.0 * K * N * N + lu_flops + 8.0 * N * N * nrhs
    bound_ms = fp64_flops / (roofline.FP64_PEAK_TFLOPS * 1e12) * 1e3
    out["fp64_path"] = {"flops": fp64_flops, "bound_ms": round(bound_ms, 2),
                        "measured_ms": round(fp64_ms, 2),
                        "frac_of_bound": round(bound_ms / fp64_ms, 4),
                        "mixed_speedup_vs_measured": round(fp64_ms / mixed_ms, 2),
                        "mixed_speedup_vs_bound": round(bound_ms / mixed_ms, 2)}
    return out


def synthesis_station(device: int, reps: int = 5) -> dict:
    """Config 4: J and dJ/dpos of the station (256 antennas x 12 MBFs, N =
    3072) through the autograd Function (forward fill + mixed solve,
    transposed solve with the cached factors, adjoint kernel), median of
    `reps` gradients timed with CUDA events after two untimed ones."""
    import torch
    from paper_1702_03781_gb300 import harp as H
    from paper_1702_03781_gb300 import synth
    from paper_1702_03781_gb300.synthesis import port_objective
    p = synth.station()
    d = torch.device("cuda", device)
    coef = torch.from_numpy(p.coef).to(d)
    sb = torch.from_numpy(p.self_blocks).to(d)
    stream = torch.cuda.current_stream()
    ms = []
    with H.Harp(device, max_N=p.N, max_nrhs=p.Na) as h:
        for i in range(2 + reps):
            x = torch.from_numpy(p.pos).to(d).requires_grad_(True)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            J = port_objective(x, h, p.freq_hz, coef, sb, prec="mixed")
            J.backward()
            e1.record(stream)
            e1.synchronize()
            if i >= 2:
                ms.append(e0.elapsed_time(e1))
    return {"N": p.N, "ports": p.Na, "ms_per_gradient": round(statistics.median(ms), 3),
            "timing": f"CUDA events around forward + backward, median of {reps} after 2"}


def synthesis_batch(device: int, ws: int, rank: int, peaks: dict, n_layouts: int = 8) -> dict:
    """Config 5's synthesis batch: J and dJ/dpos for seeded random layouts
    1..n_layouts (seeds 5001..5008) of 1024 antennas x 16 MBFs at 110 MHz
    (N = 16384, 1024 ports): forward fill + mixed solve, transposed solve
    with the cached factors, adjoint (G by exact digit products on the tensor cores). The
    layouts are sharded
    over the ranks (replicas.shard); each rank times its own with CUDA
    events (one layout per event pair) after one untimed gradient of its
    first layout; the whole job's time is the slowest rank's. The adjoint
    kernel's roofline is taken from the library's instrumentation over the
    timed layouts."""
    import torch
    from paper_1702_03781_gb300 import harp as H
    from paper_1702_03781_gb300 import replicas, roofline, synth
    from paper_1702_03781_gb300.synthesis import layout_gradients
    mine = replicas.shard(n_layouts, ws, rank)
    probs = [synth.large(1 + i) for i in mine]
    stream = torch.cuda.current_stream()
    ms, res = [], []
    prof = None
    with H.Harp(device, max_N=16384, max_nrhs=1024) as h:
        if probs:
            layout_gradients(h, probs[:1])
        torch.cuda.synchronize()
        roofline.begin(h, 1 << roofline.KINDS.index("adjoint"))
        for p in probs:
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            res += layout_gradients(h, [p])
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        prof = roofline.end(h)["adjoint"]
        digits = h.knob("adjoint_g") == 1
    total = replicas.max_over_ranks(sum(ms), torch.device("cuda", device))
    out = {"layouts": n_layouts, "seeds": [5001 + i for i in range(n_layouts)], "N": 16384,
           "ports": 1024, "ranks": ws,
           "ms_per_layout": round(total / max(1, len(probs)), 2) if probs else None,
           "job_ms": round(total, 1),
           "rank0_layouts": [5001 + i for i in mine],
           "rank0_ms": [round(m, 1) for m in ms],
           "all_converged": all(i[leg]["status"] == 0 for _, _, i in res
                                for leg in ("forward", "adjoint")),
           "corrections": {"forward": [i["forward"]["iters"] for _, _, i in res],
                           "adjoint": [i["adjoint"]["iters"] for _, _, i in res]},
           "timing": "CUDA events per layout (forward + backward), after one untimed layout"}
    if prof and prof["launches"]:
        out["adjoint_roofline"] = adjoint_roofline(prof, peaks, digits, 16384, 1024)
    return out


def adjoint_roofline(prof: dict, peaks: dict, digits: bool, N: int, nrhs: int,
                     Na: int = 1024, Nm: int = 16) -> dict:
    """The adjoint class over the timed layouts. With digit products (the
    default in the mixed modes), G = Lambda X^T and H = G C^T run as exact
    bf16 digit products: their executed flops (G: 8 Np Kp N per digit pair,
    rows padded to 128 and the right-hand sides to 64; H: 8 Na^2 128 Kts per
    digit pair, the K outputs padded to 128 and Nm^2 to 64) against the
    measured bf16 peak, beside the method's rate (8 Na (Na-1) Nm^2 (nrhs + K)
    per launch). Otherwise G runs in double-float on the FP32 pipe."""
    from paper_1702_03781_gb300 import roofline
    if not digits:
        return roofline.entry("adjoint", "ff2", prof, peaks)
    _, G, pairs = _digit_plan(nrhs)
    Np, Kp = -(-N // 128) * 128, -(-nrhs // 64) * 64
    _, _, pairs_h = _digit_plan(Nm * Nm)
    Kts = -(-(Nm * Nm) // 64) * 64
    n = max(1, prof["launches"])
    ms = prof["ms"] / n
    executed = 8.0 * Np * Kp * N * pairs + 8.0 * Na * Na * 128 * Kts * pairs_h
    _, peak, unit, note = roofline.peak_for("adjoint", "tensor_bf16", peaks)
    achieved = executed / (ms * 1e-3) / 1e12
    return {"kernel": "adjoint", "impl": "digits", "bound": "tensor",
            "achieved": round(achieved, 3), "peak": round(peak, 1), "unit": unit,
            "frac": round(achieved / peak, 4), "traffic": None, "launches": prof["launches"],
            "avg_launch_ms": round(ms, 3), "digit_pairs": pairs,
            "digit_product_flops_per_launch": executed,
            "method_flops_per_launch": prof["flops"] / n,
            "method_tflops": round(prof["flops"] / n / (ms * 1e-3) / 1e12, 3),
            "peak_source": note + " (of measured); the class also holds the slicing, the "
                                  "integer combines and the per-pair derivative sums"}


def eep_throughput(h, p, X, dev, peaks: dict, reps: int = 5) -> dict:
    """The embedded element patterns of all 256 ports of the station on the
    1-degree hemisphere grid (91 x 360 directions) from the step's solution
    (Section II-C): device time of harp_eep with CUDA events, its
    algorithmic flops (the array-factor product, 8 D Na Nm nports) against
    the TF32 tensor peak."""
    import torch
    from paper_1702_03781_gb300 import roofline
    from paper_1702_03781_gb300 import synth
    th, ph, ux, uy = synth.direction_grid(1.0, 1.0)
    F = torch.from_numpy(synth.mbf_patterns(p.Nm, th, ph, 73)).to(dev)
    pos = torch.from_numpy(p.pos).to(dev)
    uxt, uyt = torch.from_numpy(ux).to(dev), torch.from_numpy(uy).to(dev)
    E = torch.empty((2, p.Na, th.size), dtype=torch.complex64, device=dev)
    stream = torch.cuda.current_stream()
    for _ in range(2):
        h.eep(pos, p.freq_hz, X, p.Nm, uxt, uyt, F, out=E)
    ms = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        h.eep(pos, p.freq_hz, X, p.Nm, uxt, uyt, F, out=E)
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    h.sync()
    t = statistics.median(ms)
    flops = 8.0 * th.size * p.Na * p.Nm * p.Na
    _, peak, unit, note = roofline.peak_for("gemm", "tensor_tf32", peaks)
    achieved = flops / (t * 1e-3) / 1e12
    return {"directions": int(th.size), "ports": p.Na, "ms": round(t, 4),
            "flops": flops, "achieved": round(achieved, 3), "peak": round(peak, 3), "unit": unit,
            "frac": round(achieved / peak, 4), "peak_source": note + " (of measured)",
            "timing": "CUDA events around harp_eep, median of 5 after 2 warm-ups"}


def _digit_plan(K: int):
    """(digit bits b, groups G, digit pairs) of an exact-slice product over
    K terms: the widest b <= 8 with K 2^(2b-2) <= 2^24, the smallest G with
    b (G - 1) >= 53 + log2(sqrt K) + log2 G (the library's rule)."""
    import math
    b = min(8, (24 - math.ceil(math.log2(max(K, 1)))) // 2 + 1)
    G = next(g for g in range(2, 14)
             if b * (g - 1) >= 53 + 0.5 * math.log2(max(K, 1)) + math.log2(g))
    return b, G, G * (G - 1) // 2


def digit_fill(h, p, dev, peaks: dict, reps: int = 5) -> dict:
    """The FP64-accurate Z64 fill as exact digit products on the tensor
    cores (option fill64 = 1, the default inside batches of several
    contexts), timed standalone at the station: device time of its class
    (the rounds of basis digits, group products and combine; CUDA events,
    median of `reps` after 2 warm-ups), the method's rate (8 Nm^2 K per
    ordered pair) and the executed digit products (8 Np Kp per pair column
    and digit pair, rows padded to 128 and K to 64) against the bf16 peak."""
    import torch
    from paper_1702_03781_gb300 import roofline
    pos, coef, sb = (torch.from_numpy(x).to(dev) for x in (p.pos, p.coef, p.self_blocks))
    kind = roofline.KINDS.index("fill_ff")
    prev = h.knob("fill64")
    h.set_knob("fill64", 1)
    try:
        for _ in range(2):
            h.fill(pos, p.freq_hz, coef, sb, prec="mixed")
            h.z64(p.N)
        ms = []
        for _ in range(reps):
            roofline.begin(h, 1 << kind)
            h.fill(pos, p.freq_hz, coef, sb, prec="mixed")
            h.z64(p.N)
            ms.append(roofline.end(h)["fill_ff"]["ms"])
    finally:
        h.set_knob("fill64", prev)
    t = statistics.median(ms)
    K, Nm2 = p.K, p.Nm * p.Nm
    b, G, pairs = _digit_plan(K)
    Np, Kp = -(-Nm2 // 128) * 128, -(-K // 64) * 64
    method = 8.0 * Nm2 * K * p.Na * (p.Na - 1)
    executed = 8.0 * Np * Kp * (p.Na * p.Na) * pairs
    _, peak, unit, note = roofline.peak_for("residual", "tensor_bf16", peaks)
    return {"ms": round(t, 4), "method_flops": method,
            "method_tflops": round(method / (t * 1e-3) / 1e12, 3),
            "fp64_pipe_tflops": round(roofline.FP64_PEAK_TFLOPS, 3),
            "digit_bits": b, "groups": G, "digit_pairs": pairs,
            "digit_product_flops": executed,
            "digit_product_tflops": round(executed / (t * 1e-3) / 1e12, 2),
            "digit_product_frac_bf16": round(executed / (t * 1e-3) / 1e12 / peak, 4),
            "peak": round(peak, 1), "unit": unit, "peak_source": note + " (of measured)",
            "timing": "class fill_ff (CUDA events) of a standalone mixed fill with fill64 = 1, "
                      "median of 5 after 2 warm-ups"}


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def cpu_baseline(steps: int = 3, single_thread: bool = True, lapack_context: bool = True):
    """The FP64 oracle as it stands: fill + LU solve of the full station (one
    frequency per run) on this host's cores, the median of `steps` runs;
    beside it (context, not the baseline) one run of the oracle on a single
    thread, and numpy's LAPACK zgesv on the oracle's Z (median of 3)."""
    import numpy as np
    import oracle
    from paper_1702_03781_gb300 import synth
    p = synth.station()

    def run():
        t0 = time.perf_counter()
        Z = oracle.fill(p.pos, p.freq_hz, p.coef, p.self_blocks)
        oracle.solve(Z, p.V)
        return time.perf_counter() - t0, Z

    cores = oracle.num_threads()
    ts = []
    Z = None
    for _ in range(steps):
        t, Z = run()
        ts.append(t)
    out = {"value": 1e3 * statistics.median(ts), "unit": "ms", "cores": cores, "kind": "oracle",
           "runs_ms": [round(1e3 * t, 1) for t in ts],
           "sample": f"full station frequency (N=3072, 256 RHS) fill + LU solve, median of "
                     f"{steps} run(s) on {cores} threads"}
    if single_thread:
        oracle.set_threads(1)
        try:
            t1, _ = run()
        finally:
            oracle.set_threads(cores)
        out["single_thread_ms"] = round(1e3 * t1, 1)
    if lapack_context:
        tl = []
        for _ in range(3):
            t0 = time.perf_counter()
            np.linalg.solve(Z, p.V)
            tl.append(time.perf_counter() - t0)
        out["context_numpy_zgesv_ms"] = round(1e3 * statistics.median(tl), 1)
        out["context_note"] = ("numpy LAPACK zgesv of the oracle's Z for the 256 port RHS "
                               "(solve only, median of 3): a tuned CPU library for scale, "
                               "not the baseline")
    return out


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    for _ in range(args.warmup):
        cpu_baseline(1, single_thread=False, lapack_context=False)
    cb = cpu_baseline(args.steps, single_thread=False, lapack_context=False)
    line = {"impl": "reference", "metric": METRIC, "value": cb["value"], "unit": "ms",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": cb["value"], "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "l2": "n/a (CPU)"},
            "cpu_baseline": cb,
            "e2e": {"value": cb["value"], "unit": "ms", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-wideband", action="store_true")
    ap.add_argument("--no-synthesis", action="store_true",
                    help="skip the 8-layout N = 16384 synthesis batch (about a minute)")
    ap.add_argument("--pivot", default="", choices=["", "partial", "tournament", "block"],
                    help="pivot rule of the FP32 factorisation's panels (default: the library's)")
    ap.add_argument("--nvtx-step", default="",
                    help="run the warm-up, then one step of this path ('mixed' or 'fp64') inside "
                         "an NVTX range named harp_step, and exit (for an ncu launch list)")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    if args.impl == "reference":
        return run_reference(args)

    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_1702_03781_gb300 import synth
    from paper_1702_03781_gb300 import harp as H
    from paper_1702_03781_gb300 import replicas

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()

    p = synth.station()
    Na, N = p.Na, p.N
    pos = torch.from_numpy(p.pos).to(dev)
    coef = torch.from_numpy(p.coef).to(dev)
    sb = torch.from_numpy(p.self_blocks).to(dev)
    h = H.Harp(local, max_N=N, max_nrhs=Na)
    from paper_1702_03781_gb300 import autotune
    knobs = autotune.apply(h, N, p.Nm, p.K)  # the tuned tile shapes (defaults when untuned)
    if args.pivot:
        h.set_pivot(args.pivot)
    Z32 = H.colmajor_empty(N, N, torch.complex64, dev)
    Z64 = H.colmajor_empty(N, N, torch.complex128, dev)
    X = H.colmajor_empty(N, Na, torch.complex128, dev)
    X64 = H.colmajor_empty(N, Na, torch.complex128, dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # > 129 MB L2

    info = {}

    def step_mixed():
        h.fill(pos, p.freq_hz, coef, sb, prec="mixed", out=Z32)
        _, inf = h.solve(Z32, None, nrhs=Na, prec="mixed", max_iter=10, out=X)
        info.update(inf)

    def step_fp64():
        h.fill(pos, p.freq_hz, coef, sb, prec="fp64", out=Z64)
        h.solve(Z64, None, nrhs=Na, prec="fp64", out=X64)

    def barrier():
        torch.cuda.synchronize()
        replicas.barrier()
        torch.cuda.synchronize()

    def timed(fn, steps):
        ms = []
        for _ in range(steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        return ms

    from paper_1702_03781_gb300 import roofline

    if args.nvtx_step:
        fn = step_mixed if args.nvtx_step == "mixed" else step_fp64
        for _ in range(args.warmup):
            fn()
        barrier()
        torch.cuda.nvtx.range_push("harp_step")
        fn()
        torch.cuda.nvtx.range_pop()
        barrier()
        h.close()
        return 0

    for _ in range(args.warmup):
        step_mixed()
    for _ in range(2):
        step_fp64()
    barrier()
    # Device time per kernel class, one class instrumented per untimed step
    # (event pairs around many tiny launches would distort the others).
    prof_all = {}
    for kind in roofline.KINDS:
        roofline.begin(h, 1 << roofline.KINDS.index(kind))
        step_mixed()
        prof_all[kind] = roofline.end(h)[kind]
    shares = roofline.shares(prof_all)
    impl = dict(IMPL)
    if h.residual_method() == "slices":
        impl["residual"] = impl["resid_update"] = "tensor_bf16"
    # the kernel class with the most device time, whatever bounds it
    dominant = max((k for k in roofline.KINDS if prof_all[k]["launches"]),
                   key=lambda k: prof_all[k]["ms"])
    # ---- end to end through the public API with host buffers
    pos_h = torch.from_numpy(p.pos).pin_memory()
    coef_h = torch.from_numpy(p.coef).pin_memory()
    sb_h = torch.from_numpy(p.self_blocks).pin_memory()
    X_h = torch.empty((Na, N), dtype=torch.complex128).pin_memory()
    bi = pos_h.nbytes + coef_h.nbytes + sb_h.nbytes
    bo = X_h.nbytes

    def step_e2e():
        pd = pos_h.to(dev, non_blocking=True)
        cd = coef_h.to(dev, non_blocking=True)
        sd = sb_h.to(dev, non_blocking=True)
        h.fill(pd, p.freq_hz, cd, sd, prec="mixed", out=Z32)
        h.solve(Z32, None, nrhs=Na, prec="mixed", max_iter=10, out=X)
        X_h.copy_(X.T, non_blocking=True)
    for _ in range(args.warmup):
        step_e2e()

    barrier()
    L0 = H.kernel_launches()
    roofline.begin(h, 1 << roofline.KINDS.index(dominant))
    # one clock record over the three timed regions (mixed, FP64, end to end)
    with ClockSampler(local) as clk:
        barrier()
        ms_mixed = timed(step_mixed, args.steps)
        barrier()
        prof_dom = roofline.end(h)[dominant]
        L1 = H.kernel_launches()
        ms_fp64 = timed(step_fp64, max(2, min(args.steps, 5)))
        barrier()
        # agreement of the two GPU paths (last mixed step against last FP64 step)
        rel = float(torch.linalg.norm(X - X64) / torch.linalg.norm(X64))
        barrier()
        ms_e2e = timed(step_e2e, args.steps)
        barrier()

    # one frequency per rank and step: the whole job's time per frequency is
    # the slowest rank's step time over the ranks' frequencies
    t_mixed = statistics.mean(ms_mixed)
    t_max = replicas.max_over_ranks(t_mixed, dev)
    value = replicas.ms_per_unit(t_max, ws)
    e2e_max = replicas.max_over_ranks(statistics.mean(ms_e2e), dev)
    e2e_med = replicas.max_over_ranks(statistics.median(ms_e2e), dev)

    synth_batch = None
    if not args.no_synthesis:
        barrier()
        synth_batch = synthesis_batch(local, ws, rank, _peaks())

    if rank == 0:
        peaks = _peaks()
        roof = roofline.entry(dominant, impl[dominant], prof_dom, peaks)
        # every class that does arithmetic, from the untimed per-class steps
        roof_all = {k: roofline.entry(k, impl[k], prof_all[k], peaks)
                    for k in COMPUTE_KINDS + ("panel",) if prof_all[k]["launches"]}
        line = {
            "metric": METRIC, "value": round(value, 4), "unit": "ms", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(t_max, 4),
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "N": N, "nrhs": Na, "K": p.K,
                       "pivot": h.pivot_rule(), "knobs": knobs,
                       "l2": "flushed (256 MB write) before every timed step",
                       "parallelism": f"replicas x{ws}"},
            "fp64_gpu_ms_per_step": round(statistics.mean(ms_fp64), 4),
            "speedup_vs_fp64_gpu": round(statistics.mean(ms_fp64) / t_mixed, 3),
            "mixed_vs_fp64_relerr": rel,
            "refinement": {"iters": info.get("iters"), "backward_error": info.get("resid")},
            "gpu_launches": int(L1 - L0),
            "clocks": clk.summary(),
            "e2e": {"value": round(replicas.ms_per_unit(e2e_max, ws), 4), "unit": "ms",
                    "h2d_bytes_per_step": int(bi), "d2h_bytes_per_step": int(bo),
                    "median_ms": round(replicas.ms_per_unit(e2e_med, ws), 4),
                    "steps_ms": [round(m, 3) for m in ms_e2e]},
            "roofline": roof,
            "roofline_kernels": roof_all,
            "kernel_shares": shares,
        }
        # The method's own work beside the rates above (which count what the
        # kernels execute: digit products for the exact-slice residual).
        method = method_work(N, Na, p.K, prof_all, info, peaks, float(statistics.mean(ms_fp64)),
                             t_mixed)
        line["method_work"] = method
        line["eep"] = eep_throughput(h, p, X, dev, peaks)
        line["digit_fill"] = digit_fill(h, p, dev, peaks)
        if not args.no_synthesis:
            line["synthesis_station"] = synthesis_station(local)
        if synth_batch is not None:
            line["synthesis_batch"] = synth_batch
        if not args.no_wideband:
            line["wideband"] = wideband_throughput(local)
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(3)
        print(json.dumps(line))
    h.close()
    if ws > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
