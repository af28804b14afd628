"""Autotuner of the library's tile shapes and of the batch's worker count.

The knobs (context options, see include/harp_gb300.h) change how the work
is cut, never what is computed:
  * panel_rows  -- target rows per CTA of the partial-pivoting cluster panel
                   (the cluster size follows from it);
  * fill_chunk  -- the largest number of source MBFs a fill CTA stages at
                   once (0: the largest that fits shared memory);
  * splitk_max  -- the cap on the K splits of the solve's tensor-core
                   products;
  * inverses    -- where the factor inverses are built: 0 after the
                   factorisation, 1 beside it, 2 beside it unless batched;
  * fill_clusters -- GPC-sized clusters of the background FP64 fill (0:
                   about half of those the GPU holds).
For a problem class (N, Nm, K) the tuner times one mixed fill + solve of
the port excitations with CUDA events (median of a few repetitions, after
a warm-up) and walks the knobs one at a time from the defaults (coordinate
descent), keeping a change only when it is faster by more than the noise
margin. For a batch it also picks the number of worker contexts. Results
are cached as JSON, keyed by (N, Nm, K, arch).

Usage (on the GPU): python -m paper_1702_03781_gb300.autotune [--out PATH]
"""
from __future__ import annotations

import json
import os
import statistics
import sys

import torch

from . import harp as H
from . import synth

CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuned.json")
DEFAULTS = {"panel_rows": 192, "fill_chunk": 0, "splitk_max": 8, "inverses": 2,
            "fill_clusters": 0}
SPACE = {"panel_rows": [96, 128, 192, 256, 384], "fill_chunk": [0, 6, 4, 3, 2],
         "splitk_max": [8, 4, 2, 1], "inverses": [2, 0], "fill_clusters": [0, 2, 3, 5, 7]}
MARGIN = 0.01  # a change must save more than 1 % of the step


def arch() -> str:
    major, minor = torch.cuda.get_device_capability()
    return f"sm_{major}{minor}"


def key(N: int, Nm: int, K: int) -> str:
    return f"N={N},Nm={Nm},K={K},arch={arch()}"


def load(path: str = CACHE) -> dict:
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def apply(h: H.Harp, N: int, Nm: int, K: int, cache: dict | None = None) -> dict:
    """Set the cached knobs of the class (N, Nm, K) on a context (the defaults
    when the class was not tuned); returns what was set."""
    cache = load() if cache is None else cache
    knobs = dict(DEFAULTS)
    knobs.update(cache.get(key(N, Nm, K), {}).get("knobs", {}))
    for name, v in knobs.items():
        h.set_knob(name, v)
    return knobs


def _time_step(h, p, dev, reps: int) -> float:
    pos = torch.from_numpy(p.pos).to(dev)
    coef = torch.from_numpy(p.coef).to(dev)
    sb = torch.from_numpy(p.self_blocks).to(dev)
    Z = H.colmajor_empty(p.N, p.N, torch.complex64, dev)
    X = H.colmajor_empty(p.N, p.Na, torch.complex128, dev)
    stream = torch.cuda.current_stream()

    def step():
        h.fill(pos, p.freq_hz, coef, sb, prec="mixed", out=Z)
        h.solve(Z, None, nrhs=p.Na, prec="mixed", out=X)

    step()
    ms = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    return statistics.median(ms)


def tune_problem(p, device: int = 0, reps: int = 3, log=None) -> dict:
    """Coordinate descent over the knobs for one problem (fill + mixed solve
    of its port excitations); returns {"knobs", "ms", "default_ms", "trials"}."""
    dev = torch.device("cuda", device)
    trials = []
    with H.Harp(device, max_N=p.N, max_nrhs=p.Na) as h:
        cur = dict(DEFAULTS)
        for name, v in cur.items():
            h.set_knob(name, v)
        best = base = _time_step(h, p, dev, reps)
        trials.append({"knobs": dict(cur), "ms": round(base, 4)})
        for name, values in SPACE.items():
            for v in values:
                if v == cur[name] or (name == "fill_chunk" and v > p.Nm):
                    continue
                h.set_knob(name, v)
                t = _time_step(h, p, dev, reps)
                trials.append({"knobs": dict(cur, **{name: v}), "ms": round(t, 4)})
                if log:
                    log(f"  {name}={v}: {t:.3f} ms (best {best:.3f})")
                if t < best * (1 - MARGIN):
                    best, cur[name] = t, v
            h.set_knob(name, cur[name])
    return {"knobs": cur, "ms": round(best, 4), "default_ms": round(base, 4), "trials": trials}


def tune_batch_workers(problems, device: int = 0, candidates=(2, 3, 4, 6), cache=None,
                       log=None) -> dict:
    """The number of worker contexts, where they build their factor inverses
    (after the factorisation, or beside it on two more streams) and how
    their background FP64 fill runs (digit products on the tensor cores, or
    the float-float kernel) for a batch of problems: device time of one
    batch call after a warm-up batch, each context's other knobs from the
    cache for the batch's median problem class."""
    cache = load() if cache is None else cache
    dev = f"cuda:{device}"
    items = [H.BatchItem(torch.from_numpy(q.pos).to(dev), q.freq_hz,
                         torch.from_numpy(q.coef).to(dev), torch.from_numpy(q.self_blocks).to(dev))
             for q in problems]
    max_N = max(it.N for it in items)
    mid = sorted(problems, key=lambda q: q.N)[len(problems) // 2]
    res = {}
    for n in candidates:
        for inv in (2, 1):
            for f64 in (2, 0):
                ctxs = [H.Harp(device, max_N=max_N, max_nrhs=256) for _ in range(n)]
                for c in ctxs:
                    apply(c, mid.N, mid.Nm, mid.K, cache)
                    c.set_knob("inverses", inv)
                    c.set_knob("fill64", f64)
                H.solve_batch(ctxs, items[-n:], prec="mixed")
                H.solve_batch(ctxs, items, prec="mixed", check=False)
                res[(n, inv, f64)] = ctxs[0].batch_device_ms() / len(items)
                if log:
                    log(f"  workers={n} inverses={inv} fill64={f64}: "
                        f"{res[(n, inv, f64)]:.3f} ms per problem")
                for c in ctxs:
                    c.close()
    best = min(res, key=res.get)
    return {"workers": best[0], "inverses": best[1], "fill64": best[2],
            "ms_per_problem": round(res[best], 4),
            "trials": {f"{k[0]}x{k[1]}x{k[2]}": round(v, 4) for k, v in res.items()},
            "class": key(mid.N, mid.Nm, mid.K)}


def main(argv=None) -> int:
    import argparse
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=CACHE)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--batch-only", action="store_true",
                    help="retune only the wideband batch's workers, keeping the cached classes")
    args = ap.parse_args(argv)
    from . import build
    build.build()
    log = lambda s: print(s, file=sys.stderr, flush=True)  # noqa: E731
    cache = load(args.out)
    wb = synth.wideband()
    mid = sorted(wb, key=lambda q: q.N)[len(wb) // 2]  # the class the batch's contexts use
    classes = [] if args.batch_only else [synth.station(), mid] + [wb[i] for i in (0, 21, 42, 63)]
    for p in classes:
        log(f"tuning {p.name} (N={p.N}, Nm={p.Nm}, K={p.K})")
        cache[key(p.N, p.Nm, p.K)] = tune_problem(p, reps=args.reps, log=log)
    log("tuning the wideband batch's workers")
    cache["wideband_batch"] = tune_batch_workers(wb, cache=cache, log=log)
    with open(args.out, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    log(f"wrote {args.out}")
    return 0


if __name__ == "__main__":
    sys.exit(main())
