"""Autotuner for the library's launch shapes (qdwhp_tune_set), per size class.

The library reads three launch parameters from a per-size-class table (see include/qdwhp.h):
the rows per CTA of the cooperative Householder panel, the least warps per CTA of a Jacobi
sweep, and the CTAs per SM that split-K aims for.  Every value computes the same result, so
tuning is a matter of timing.  For each class, smallest first, `tune` times QDWHpartial-EIG
(top 10 %, eigenvalues uniform in [-1, 1]) at a representative order on the device for every
candidate of every knob in turn, keeping the fastest (coordinate descent), and returns the
table.  The objective is the use the table serves: "latency" times one solve at a time (CUDA
events, median of `reps` after a warm-up); "throughput" times a batch of `batch` solves
through qdwhp_eig_batched at `concurrency` worker streams (median wall time).  The two
objectives pick different tables (alone, a solve ran fastest with 32-row panel slices in
every class).  Larger solves reach into smaller classes (their trailing panels and reduced
problems), which is why the small classes are settled first.  `save`/`load` keep the table
as JSON; `apply` installs it.

Measured on the batched workload (512 solves, n in [64, 1024], 16 worker streams): neither
objective's table beat the built-in defaults (44.4-44.8 solves/s; latency-tuned 38.4,
throughput-tuned 41.6).  A class is tuned on one order and one matrix, while the batch mixes
sizes whose solves overlap, and two timed batches per candidate sit within the run-to-run
spread.  The defaults stay; the tuner is a tool for other workloads and devices.
"""

from __future__ import annotations

import json
import statistics

KNOBS = {
    "panel_rows_per_cta": (0, (32, 64, 128, 256)),
    "jacobi_min_warps": (1, (1, 2, 4, 8)),
    "splitk_ctas_per_sm": (2, (1, 2, 4)),
}
# representative order of each size class (<= 128, <= 256, <= 512, <= 1024, larger)
CLASS_ORDERS = (96, 192, 384, 768, 1536)


def _time_solve(Q, A, k, reps: int) -> float:
    import torch
    Q.eig(A, k=k)
    torch.cuda.synchronize()
    out = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        Q.eig(A, k=k)
        e1.record()
        torch.cuda.synchronize()
        out.append(e0.elapsed_time(e1))
    return statistics.median(out)


def _time_batch(Q, A, batch: int, concurrency: int, reps: int) -> float:
    import time

    import torch
    As = [A] * batch
    Q.eig_batched(As[: max(1, concurrency)], 0.10, concurrency=concurrency)
    torch.cuda.synchronize()
    out = []
    for _ in range(reps):
        t0 = time.perf_counter()
        _, sts = Q.eig_batched(As, 0.10, concurrency=concurrency)
        torch.cuda.synchronize()
        out.append(1e3 * (time.perf_counter() - t0))
        if any(sts):
            raise RuntimeError(f"a tuning solve failed: {sts}")
    return statistics.median(out)


def tune(classes=(0, 1, 2, 3, 4), reps: int = 5, seed: int = 5150, objective: str = "latency",
         batch: int = 32, concurrency: int = 16) -> dict:
    """Times the candidates on the current CUDA device; returns the table (and the timings)."""
    if objective not in ("latency", "throughput"):
        raise ValueError("objective is 'latency' or 'throughput'")
    from . import build
    build.build()
    from . import inputs as I
    from . import qdwhp as Q

    lib = Q.lib()
    table = {name: [lib.qdwhp_tune_get(knob, c) for c in range(5)] for name, (knob, _) in KNOBS.items()}
    log = []
    for c in classes:
        n = CLASS_ORDERS[c]
        A, _, k = I.eig_uniform_device(n, seed + c, 0.10)
        for name, (knob, cands) in KNOBS.items():
            best_v, best_t = None, float("inf")
            for v in cands:
                if lib.qdwhp_tune_set(knob, c, v) != 0:
                    continue
                t = _time_solve(Q, A, k, reps) if objective == "latency" else \
                    _time_batch(Q, A, batch, concurrency, reps)
                log.append({"class": c, "n": n, "knob": name, "value": v, "ms": t})
                if t < best_t:
                    best_v, best_t = v, t
            lib.qdwhp_tune_set(knob, c, best_v)
            table[name][c] = best_v
    return {"version": 1, "objective": objective, "classes": ["<=128", "<=256", "<=512", "<=1024", ">1024"],
            "table": table, "log": log}


def apply(result: dict) -> None:
    """Installs a table produced by `tune` (or read by `load`)."""
    from . import qdwhp as Q
    lib = Q.lib()
    for name, values in result["table"].items():
        knob = KNOBS[name][0]
        for c, v in enumerate(values):
            if lib.qdwhp_tune_set(knob, c, int(v)) != 0:
                raise ValueError(f"{name}[{c}] = {v} is outside the knob's range")


def save(result: dict, path: str) -> None:
    with open(path, "w") as f:
        json.dump(result, f, indent=1)


def load(path: str) -> dict:
    with open(path) as f:
        result = json.load(f)
    if result.get("version") != 1 or set(result.get("table", {})) != set(KNOBS):
        raise ValueError(f"{path} is not a version-1 tuning table")
    for name, values in result["table"].items():
        if len(values) != 5:
            raise ValueError(f"{path}: {name} needs one value per size class")
    return result
