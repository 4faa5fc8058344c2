#!/usr/bin/env python3
"""Throughput of QDWHpartial-SVD on one GB300 (and replicas on N GPUs).

Workload (one step = one full solve): A = U diag(sigma) V^T, 4096 x 4096, FP64,
Haar U and V, sigma_i = 10^(-12 i / 4095); the 5 % largest singular triplets
(k = 205).  Every step runs the whole hot path: Lanczos norm estimate,
count-to-threshold subspace, QDWH iterations, extraction QR, index rule, Q2,
A Q2 and its SVD, back-transform.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

`--impl reference` times the FP64 CPU oracle on the host cores (the method's
plain CPU implementation, test infrastructure) on the same workload.
For N > 1 (launched by torchrun) every rank solves its own independent problem
(replicas, no collective on the data path); the value is all ranks' solves over
the slowest rank's time.
"""

from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "partial EIG/SVD solves/sec and TFLOP/s vs FP64/TF32 peak; p50/p99 latency, mixed vs FP64"
UNIT = "solves/s"
M = N = 4096
FRACTION = 0.05
SEED = 2000
L2_FLUSH_BYTES = 256 << 20

# Roofline denominator for FP64 DMMA: no FP64 figure is in the measured-peaks file, so it is the
# measured BF16 dense burst peak times the nominal FP64 / BF16 ratio (1.25 TFLOP/s / 2250 TFLOP/s).
NOMINAL_FP64_OVER_BF16 = 1.25 / 2250.0


def workload_config(k):
    return {"workload": f"QDWHpartial-SVD {M}x{N} FP64, sigma log-spaced 1..1e-12, top 5% (k={k})",
            "m": M, "n": N, "k": k, "seed": SEED,
            "l2": "L2 flushed (256 MB write) between timed steps; A alone is 134 MB > L2"}


def svd_flops(m, n, ell, k, it_qr, it_chol):
    """Algorithmic flops of one solve: QDWH steps (Cholesky: 3mn^2 + n^3/3; QR: 2(2(m+n)n^2 - 2n^3/3) + 2mn^2),
    I - X^T X (mn^2), Householder QR (4/3 n^3), Q2 (2 n^2 ell), A Q2 (2 m n ell), reduced SVD (4 m ell^2 +
    17 ell^3) and V = Q2 V~ (2 n ell k)."""
    f = it_chol * (3.0 * m * n * n + n ** 3 / 3.0)
    f += it_qr * (2.0 * (2.0 * (m + n) * n * n - 2.0 * n ** 3 / 3.0) + 2.0 * m * n * n)
    f += m * n * n + 4.0 / 3.0 * n ** 3 + 2.0 * n * n * ell + 2.0 * m * n * ell + 4.0 * m * ell ** 2
    f += 17.0 * ell ** 3 + 2.0 * n * ell * k
    return f


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi samples during the timed region."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 8:
                self.rows.append(parts)

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        if self.thread is not None:
            self.thread.join(timeout=5)
        sm = []
        smax = None
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[0]))
                smax = float(r[1])
            except ValueError:
                continue
            for nm, v in zip(names, r[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def make_problem(seed):
    from paper_2104_14186_gb300 import inputs as I
    return I.svd_logspaced(M, N, seed, FRACTION)


def oracle_solve(A, k):
    import oracle as O
    return O.qdwhp_svd(A, O.SvdOptions(k=k))


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if args.impl == "ours" else "gloo")
    return world, rank, local


def replica_seed(rank):
    """Each rank solves its own replica of the workload (independent problems, no collective)."""
    return SEED + rank


def max_over_ranks(value, world, device):
    """The slowest rank's time (the contract's max-over-ranks), a no-op for one rank."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_rate(world, steps, total_ms):
    """Whole-job throughput: every rank's solves over the slowest rank's time."""
    return world * steps / (total_ms / 1e3)


def run_reference(args):
    world, rank, _ = dist_setup(args)
    if rank != 0:
        return
    import numpy as np  # noqa: F401
    p = make_problem(SEED)
    cores = os.cpu_count()
    for _ in range(args.warmup):
        oracle_solve(p.A, p.k)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle_solve(p.A, p.k)
        times.append(time.perf_counter() - t0)
    total = sum(times)
    value = args.steps / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(p.k),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{args.steps} full solves of the {M}x{N} workload (numpy/LAPACK FP64 oracle)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_ours(args):
    import numpy as np
    import torch

    world, rank, local = dist_setup(args)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2104_14186_gb300 import build
    build.build()
    from paper_2104_14186_gb300 import qdwhp as Q

    p = make_problem(replica_seed(rank))
    # host copy in column-major storage (the layout the C ABI takes), page-locked
    A_host = torch.from_numpy(np.ascontiguousarray(p.A.T)).pin_memory().t()
    A = torch.from_numpy(np.ascontiguousarray(p.A)).to(dev)
    k = p.k
    sopts = {"precision": precision_code(Q, args.precision), "refine_steps": args.refine, "zolo_r": args.zolo}
    o = Q.default_opts(**sopts)
    ctypes = __import__("ctypes")
    ws = Q.workspace(Q.lib().qdwhp_svd_workspace_bytes(M, N, ctypes.byref(o)), dev)
    ws_host = Q.workspace(Q.lib().qdwhp_svd_host_workspace_bytes(M, N, k, ctypes.byref(o)), dev)
    host_out = (torch.empty(k, dtype=torch.float64, pin_memory=True),
                torch.empty(k, M, dtype=torch.float64, pin_memory=True),
                torch.empty(k, N, dtype=torch.float64, pin_memory=True))
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    for _ in range(args.warmup):
        r = Q.svd(A, k=k, ws=ws, **sopts)
    torch.cuda.synchronize()

    # ---- timed region: inputs resident in HBM ----
    sampler = ClockSampler(local)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    barrier()
    torch.cuda.synchronize()
    sampler.start()
    launches0 = Q.launch_count()
    infos = []
    for i in range(args.steps):
        flush.zero_()
        ev[i][0].record(stream)
        r = Q.svd(A, k=k, ws=ws, **sopts)
        ev[i][1].record(stream)
        infos.append(r.info)
    torch.cuda.synchronize()
    barrier()
    launches = Q.launch_count() - launches0
    clocks = sampler.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = max_over_ranks(sum(step_ms), world, dev)
    value = aggregate_rate(world, args.steps, total_ms)

    # ---- roofline pass: the same solves with every GEMM launch bracketed by CUDA events on its
    # stream (kept out of the timed region above, whose value carries no instrumentation) ----
    prof_steps = max(1, min(3, args.steps))
    pev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(prof_steps)]
    Q.profile_begin()
    for i in range(prof_steps):
        flush.zero_()
        pev[i][0].record(stream)
        Q.svd(A, k=k, ws=ws, **sopts)
        pev[i][1].record(stream)
    torch.cuda.synchronize()
    prof = Q.profile_end()
    prof_total_ms = sum(a.elapsed_time(b) for a, b in pev)

    # ---- end to end through the C ABI's host-buffer entry (qdwhp_svd_host: the H2D copy of A and
    # the D2H copies of sigma, U, V run on the stream inside the call) ----
    e2e_ms = []
    for i in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        rh = Q.svd(A_host, k=k, ws=ws_host, device=dev, out=host_out, **sopts)
        e2e_ms.append(1e3 * (time.perf_counter() - t0))
    e2e_total = max_over_ranks(sum(e2e_ms), world, dev)
    h2d = M * N * 8
    d2h = (rh.sigma.numel() + rh.U.numel() + rh.V.numel()) * 8

    info = infos[-1]
    fl = svd_flops(M, N, info["ell"], k, info["it_qr"], info["it_chol"])
    # accuracy of this result against sigma* and the residuals (FP64, outside the timed region)
    sig_true = torch.from_numpy(p.sigma[:k]).to(dev)
    nA = torch.linalg.norm(A)
    acc = {"sigma_err": (torch.max(torch.abs(r.sigma - sig_true)) / sig_true[0]).item(),
           "residV": (torch.linalg.norm(A @ r.V - r.U * r.sigma[None, :]) / nA).item(),
           "residU": (torch.linalg.norm(A.T @ r.U - r.V * r.sigma[None, :]) / nA).item(),
           "orthU": torch.linalg.norm(r.U.T @ r.U - torch.eye(k, dtype=torch.float64, device=dev)).item(),
           "orthV": torch.linalg.norm(r.V.T @ r.V - torch.eye(k, dtype=torch.float64, device=dev)).item()}
    peaks = load_peaks()
    bf16 = peaks.get("bf16_tflops")
    peak = bf16 * NOMINAL_FP64_OVER_BF16 if bf16 else 1.9e3 * NOMINAL_FP64_OVER_BF16
    # the DMMA kernel's own launches (records with split-K slices >= 1; -1 and -2 mark the
    # tensor-core products of the emulated and mixed precisions)
    dmma = [r for r in Q.profile_records() if r[4] >= 1]
    dmma_ms = sum(r[5] for r in dmma)
    dmma_flops = sum((r[1] * (r[1] + 1) * r[2]) if r[3] else 2.0 * r[0] * r[1] * r[2] for r in dmma)
    achieved = dmma_flops / (dmma_ms / 1e3) / 1e12 if dmma_ms > 0 else None
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": DTYPES[args.precision],
        "data": "synthetic", "config": workload_config(k),
        "mode": {"precision": args.precision, "refine_steps": args.refine,
                 "polar": "zolo-pd r=%d" % args.zolo if args.zolo else "qdwh"},
        "accuracy": acc,
        "tflops": fl / (total_ms / args.steps / 1e3) / 1e12,
        "tflops_frac_of_fp64_peak": fl / (total_ms / args.steps / 1e3) / 1e12 / peak,
        "solve": {"ell": info["ell"], "it_qr": info["it_qr"], "it_chol": info["it_chol"], "s": info["s"],
                  "alpha": info["alpha"], "jacobi_sweeps": info["jacobi_sweeps"], "alg_flops": fl,
                  "step_ms": step_ms},
        "roofline": {
            "kernel": "dgemm_kernel (FP64 DMMA mma.sync m8n8k4 tiles, all GEMM/SYRK/TRSM/QR-update launches)",
            "bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": (achieved / peak) if achieved else None,
            # DRAM bytes of one 4096^3 launch from the ncu capture in profiles/ (the kernel is unchanged)
            "traffic": DGEMM_4096_TRAFFIC_BYTES, "traffic_launch": "dgemm_kernel<32,32,0,0> 4096^3",
            "peak_source": "measured bf16 dense burst x nominal FP64/BF16 ratio (1.25/2250), of measured",
            "gemm_share_of_step": dmma_ms / prof_total_ms if prof_total_ms > 0 else None,
            "gemm_launches_per_solve": len(dmma) / prof_steps,
            "measured": f"CUDA events around every GEMM launch in {prof_steps} instrumented solves run after "
                        "the timed steps (same workload, workspace and stream)",
        },
        "e2e": {"value": aggregate_rate(world, args.steps, e2e_total), "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": int(launches),
        "clocks": clocks,
    }
    if args.precision in ("emulated", "mixed-emulated"):
        line["all_products_fp64_equivalent"] = line["roofline"]
        line["roofline"] = emulated_roofline(Q, prof_total_ms, bf16 if bf16 else 1.9e3)
    if args.precision in ("mixed", "mixed-emulated"):
        key = "roofline" if args.precision == "mixed" else "roofline_fp32_products"
        if args.precision == "mixed":
            line["fp64_products"] = line["roofline"]
        line[key] = bf16x6_roofline(Q, prof_total_ms, bf16 if bf16 else 1.9e3)
    if args.precision == "fp64" and not args.no_variants:
        line["variants"] = precision_variants(Q, A, k, p, dev, flush, stream)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        t0 = time.perf_counter()
        oracle_solve(p.A, k)
        dt = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": 1.0 / dt, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                                "sample": f"1 full solve of the {M}x{N} workload (numpy/LAPACK FP64 oracle)"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def precision_variants(Q, A, k, p, dev, flush, stream, steps=3, warmup=2):
    """The same workload in the other precision modes (a few timed solves each, after the
    headline's timed region): emulated FP64 products, and FP32 Cholesky steps + emulated
    products + 6 FP64 refinement steps on Q2 (both at the plain-FP64 tolerances), with their
    accuracy against sigma* and the residuals."""
    import torch
    out = {}
    sig_true = torch.from_numpy(p.sigma[:k]).to(dev)
    nA = torch.linalg.norm(A)
    for name, opts in (("emulated", {"precision": Q.FP64_EMULATED}),
                       ("mixed-emulated", {"precision": Q.MIXED_EMULATED, "refine_steps": 6})):
        o = Q.default_opts(**opts)
        ws = Q.workspace(Q.lib().qdwhp_svd_workspace_bytes(M, N, __import__("ctypes").byref(o)), dev)
        for _ in range(warmup):
            r = Q.svd(A, k=k, ws=ws, **opts)
        torch.cuda.synchronize()
        ms = []
        for _ in range(steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            r = Q.svd(A, k=k, ws=ws, **opts)
            e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        t = statistics.median(ms)
        out[name] = {"value": 1e3 / t, "unit": UNIT, "ms_per_step": t, "steps": steps, "options": {
                         kk: int(v) for kk, v in opts.items()},
                     "accuracy": {"sigma_err": (torch.max(torch.abs(r.sigma - sig_true)) / sig_true[0]).item(),
                                  "residV": (torch.linalg.norm(A @ r.V - r.U * r.sigma[None, :]) / nA).item(),
                                  "residU": (torch.linalg.norm(A.T @ r.U - r.V * r.sigma[None, :]) / nA).item()}}
        del ws
    return out


def precision_code(Q, name):
    return {"fp64": Q.FP64, "mixed": Q.MIXED, "emulated": Q.FP64_EMULATED, "mixed-emulated": Q.MIXED_EMULATED}[name]


DTYPES = {"fp64": "f64", "mixed": "f32+f64", "emulated": "f64 (bf16 Ozaki digit products + f64 sums)",
          "mixed-emulated": "f32 + f64 (bf16 Ozaki digit products + f64 sums)"}
OZ_PAIRS = 60          # digit products per emulated FP64 product
DGEMM_4096_TRAFFIC_BYTES = 1.347e9   # dram read + write of one 4096^3 dgemm_kernel launch (ncu)


def emulated_roofline(Q, total_ms, bf16_peak):
    """Roofline of the emulated-product kernel from the per-GEMM records (split slot -1):
    its own arithmetic is BF16 tensor work, 60 digit products of each FP64 product.  The
    count is algorithmic (the unpadded shape; n(n+1)k for a lower SYRK), not what the
    128 x 128 x 64-padded tiles issue."""
    recs = [r for r in Q.profile_records() if r[4] < 0]
    if not recs:
        return None
    ms = sum(r[5] for r in recs)
    fp64_flops = sum((r[1] * (r[1] + 1) * r[2]) if r[3] else 2.0 * r[0] * r[1] * r[2] for r in recs)
    bf16_flops = OZ_PAIRS * fp64_flops
    achieved = bf16_flops / (ms / 1e3) / 1e12
    return {"kernel": "oz_umma_kernel (FP64 products as 60 exact BF16 digit products in 2x2 digit blocks, tcgen05.mma kind::f16, "
                      "FP32 sums in TMEM)",
            "bound": "tensor", "achieved": achieved, "peak": bf16_peak, "unit": "TFLOP/s",
            "frac": achieved / bf16_peak, "traffic": None,
            "peak_source": "measured bf16 dense burst (cuBLAS), of measured",
            "fp64_equivalent_tflops": fp64_flops / (ms / 1e3) / 1e12,
            "share_of_step": ms / total_ms, "launches": len(recs)}


B6_PAIRS = 6          # BF16 slice products per FP32-accurate product


def bf16x6_roofline(Q, total_ms, bf16_peak):
    """Roofline of the FP32-accurate BF16x6 kernel from the per-GEMM records (split slot -2): its
    arithmetic is BF16 tensor work, six slice products of each FP32 product (algorithmic count of
    the unpadded shape)."""
    recs = [r for r in Q.profile_records() if r[4] == -2]
    if not recs:
        return None
    ms = sum(r[5] for r in recs)
    fp32_flops = sum((r[1] * (r[1] + 1) * r[2]) if r[3] else 2.0 * r[0] * r[1] * r[2] for r in recs)
    achieved = B6_PAIRS * fp32_flops / (ms / 1e3) / 1e12
    return {"kernel": "b6_umma_kernel (FP32 products as 6 BF16 slice products, tcgen05.mma kind::f16, FP32 sums in "
                      "TMEM)",
            "bound": "tensor", "achieved": achieved, "peak": bf16_peak, "unit": "TFLOP/s",
            "frac": achieved / bf16_peak, "traffic": None,
            "peak_source": "measured bf16 dense burst (cuBLAS), of measured",
            "fp32_equivalent_tflops": fp32_flops / (ms / 1e3) / 1e12,
            "share_of_step": ms / total_ms, "launches": len(recs)}


def run_kernel_gemm(args):
    """Isolated DMMA GEMM C = A B (4096^3, FP64) through qdwhp_gemm_f64, one launch per step."""
    import torch

    from paper_2104_14186_gb300 import build
    build.build()
    from paper_2104_14186_gb300 import qdwhp as Q

    n = 4096
    g = torch.Generator(device="cuda").manual_seed(1)
    A = torch.randn(n, n, dtype=torch.float64, device="cuda", generator=g)
    B = torch.randn(n, n, dtype=torch.float64, device="cuda", generator=g)
    Cm = torch.empty(n, n, dtype=torch.float64, device="cuda")
    st = torch.cuda.current_stream()
    lib = Q.lib()

    emulated = args.precision == "emulated"
    fp32 = args.precision == "mixed"
    ws = Q.workspace(lib.qdwhp_gemm_f64_emulated_workspace_bytes(n, n, n)) if emulated else None
    if fp32:
        A, B, Cm = A.float(), B.float(), Cm.float()
        ws = Q.workspace(lib.qdwhp_gemm_f32_bf16x6_workspace_bytes(n, n, n))

    def step():
        if fp32:
            rc = lib.qdwhp_gemm_f32_bf16x6(0, 0, n, n, n, 1.0, A.data_ptr(), n, B.data_ptr(), n, 0.0,
                                           Cm.data_ptr(), n, ws.data_ptr(), ws.numel(), st.cuda_stream)
        elif emulated:
            rc = lib.qdwhp_gemm_f64_emulated(0, 0, n, n, n, 1.0, A.data_ptr(), n, B.data_ptr(), n, 0.0,
                                             Cm.data_ptr(), n, ws.data_ptr(), ws.numel(), st.cuda_stream)
        else:
            rc = lib.qdwhp_gemm_f64(0, 0, n, n, n, 1.0, A.data_ptr(), n, B.data_ptr(), n, 0.0, Cm.data_ptr(), n,
                                    st.cuda_stream)
        assert rc == 0

    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    ms = []
    for _ in range(args.steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        step()
        e1.record(st)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    peaks = load_peaks()
    peak = peaks.get("bf16_tflops", 1.9e3) * NOMINAL_FP64_OVER_BF16
    tf = 2.0 * n ** 3 / (statistics.median(ms) / 1e3) / 1e12
    if fp32:
        bf16_peak = peaks.get("bf16_tflops", 1.9e3)
        bf16_tf = B6_PAIRS * 2.0 * n ** 3 / (statistics.median(ms) / 1e3) / 1e12
        print(json.dumps({"kernel": "b6 split + b6_umma_kernel via qdwhp_gemm_f32_bf16x6", "m": n, "n": n, "k": n,
                          "ms_median": statistics.median(ms), "fp32_equivalent_tflops": tf, "bf16_tflops": bf16_tf,
                          "bf16_peak": bf16_peak, "bf16_frac": bf16_tf / bf16_peak}), flush=True)
        return
    if emulated:
        bf16_peak = peaks.get("bf16_tflops", 1.9e3)
        bf16_tf = OZ_PAIRS * 2.0 * n ** 3 / (statistics.median(ms) / 1e3) / 1e12
        print(json.dumps({"kernel": "oz split + oz_umma_kernel via qdwhp_gemm_f64_emulated", "m": n, "n": n, "k": n,
                          "ms_median": statistics.median(ms), "fp64_equivalent_tflops": tf,
                          "vs_fp64_peak": tf / peak, "bf16_tflops": bf16_tf, "bf16_peak": bf16_peak,
                          "bf16_frac": bf16_tf / bf16_peak}), flush=True)
        return
    print(json.dumps({"kernel": "dgemm_kernel<32,32,N,N> via qdwhp_gemm_f64", "m": n, "n": n, "k": n,
                      "ms_median": statistics.median(ms), "tflops": tf, "peak": peak, "frac": tf / peak,
                      "alg_bytes": 3 * n * n * 8}), flush=True)


def run_eig_large(args):
    """The n = 16384 EIG workload (clustered spectrum), 1 % or 20 % largest, timed per solve, for
    each precision of --precisions (default: --precision); with --cpu-baseline the FP64 oracle is
    timed once on the host cores on the same matrix."""
    import numpy as np
    import torch

    from paper_2104_14186_gb300 import build
    build.build()
    from paper_2104_14186_gb300 import inputs as I
    from paper_2104_14186_gb300 import qdwhp as Q

    frac = args.fraction
    A, lam, k = I.eig_clustered_device(16384, 3000, frac)
    n = A.shape[0]
    peak = load_peaks().get("bf16_tflops", 1.9e3) * NOMINAL_FP64_OVER_BF16
    true = np.sort(lam)[::-1][:k]
    nA = torch.linalg.norm(A)
    for name in (args.precisions.split(",") if args.precisions else [args.precision]):
        prec = precision_code(Q, name)
        o = Q.default_opts(precision=prec, zolo_r=args.zolo)
        ws = Q.workspace(Q.lib().qdwhp_eig_workspace_bytes(n, __import__("ctypes").byref(o)))
        for _ in range(args.warmup):
            r = Q.eig(A, k=k, ws=ws, precision=prec, zolo_r=args.zolo)
        torch.cuda.synchronize()
        ms = []
        for _ in range(args.steps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            r = Q.eig(A, k=k, ws=ws, precision=prec, zolo_r=args.zolo)
            e1.record()
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        # GEMM share from one instrumented solve after the timed ones
        Q.profile_begin()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        Q.eig(A, k=k, ws=ws, precision=prec, zolo_r=args.zolo)
        e1.record()
        torch.cuda.synchronize()
        prof = Q.profile_end()
        prof_ms = e0.elapsed_time(e1)
        err = float(np.max(np.abs(r.lam.cpu().numpy() - true)))
        V = r.V
        res = (torch.linalg.norm(A @ V - V * r.lam[None, :]) / nA).item()
        orth = torch.linalg.norm(V.T @ V - torch.eye(k, dtype=torch.float64, device=V.device)).item()
        ell = r.info["ell"]
        fl = 3 * (n ** 3 + n ** 3 / 3 + 2 * n ** 3) + 4 / 3 * n ** 3 + 4 * n * n * ell + 2 * n * ell ** 2 \
            + 9 * ell ** 3 + 2 * n * ell * k
        t = statistics.median(ms) / 1e3
        del ws
        line = {"workload": f"QDWHpartial-EIG n={n} clustered, {100 * frac:g}% largest (k={k})",
                "precision": name, "zolo_r": args.zolo, "ell": ell, "ms_median": 1e3 * t, "steps": args.steps,
                "solves_per_s": 1 / t, "alg_tflops": fl / t / 1e12, "alg_frac_of_fp64_peak": fl / t / 1e12 / peak,
                "fp64_peak_tflops": peak,
                "gemm_tflops": prof["gemm_flops"] / prof["gemm_ms"] * 1e-9 if prof["gemm_ms"] else None,
                "gemm_share": prof["gemm_ms"] / prof_ms, "lam_err": err / float(np.max(np.abs(lam))),
                "resid": res, "orth": orth, "jacobi_sweeps": r.info["jacobi_sweeps"], "dc_nodes": r.info["dc_nodes"],
                "it_f32": r.info["it_f32"]}
        print(json.dumps(line), flush=True)
    if args.cpu_baseline:
        # Bounded sample of the FP64 oracle on the host cores: its first Cholesky-based QDWH step
        # (eq. practical-polar-chol, 10/3 n^3 flops) on this matrix, shifted and scaled as the
        # solver does, scaled to one solve by the algorithmic flop count (a full solve at this
        # size takes tens of minutes on the host).
        import oracle as O
        X = A.cpu().numpy()
        del A
        torch.cuda.empty_cache()
        t_thr, mu = r.info["t"], r.info["mu"]      # A' = -A, B = A' + t I (units of A), mu = lambda_min(B)
        s_eig = 0.2
        X *= -(1.0 - s_eig) / abs(mu)
        X[np.diag_indices(n)] += (1.0 - s_eig) * t_thr / abs(mu) - s_eig
        a, b, c, _ = O.dwh_weights(s_eig)
        t0 = time.perf_counter()
        O.qdwh_chol_step(X, a, b, c)
        dt = time.perf_counter() - t0
        per_solve = dt * fl / (10.0 / 3.0 * n ** 3)
        print(json.dumps({"workload": f"QDWHpartial-EIG n={n} clustered, {100 * frac:g}% largest (k={k})",
                          "cpu_baseline": {"value": 1.0 / per_solve, "unit": "solves/s", "cores": os.cpu_count(),
                                           "kind": "oracle", "sample_seconds": dt,
                                           "sample": "one Cholesky-based QDWH step of the numpy/LAPACK FP64 oracle "
                                                     f"on this n={n} matrix (10/3 n^3 flops), scaled to a solve by the "
                                                     f"algorithmic flop count of the GPU run (ell={ell})"}}),
              flush=True)


def run_gesvd(args):
    """Full-spectrum QDWH-SVD (every triplet) of the 4096 x 4096 workload (sigma log-spaced
    1 .. 1e-12), timed per solve; FP64 or emulated FP64 products."""
    import torch

    from paper_2104_14186_gb300 import build
    build.build()
    from paper_2104_14186_gb300 import qdwhp as Q

    if args.precision not in ("fp64", "emulated"):
        raise SystemExit("--gesvd takes --precision fp64 or emulated")
    prec = precision_code(Q, args.precision)
    p = make_problem(2000)
    A = torch.from_numpy(p.A).to("cuda")
    m, n = A.shape
    ws = Q.workspace(Q.lib().qdwhp_gesvd_workspace_bytes(m, n, prec))
    for _ in range(args.warmup):
        s, U, V, info = Q.gesvd(A, precision=prec, ws=ws)
    torch.cuda.synchronize()
    ms = []
    Q.profile_begin()
    for _ in range(args.steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        s, U, V, info = Q.gesvd(A, precision=prec, ws=ws)
        e1.record()
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    prof = Q.profile_end()
    sig = torch.from_numpy(p.sigma).to("cuda")
    nA = torch.linalg.norm(A)
    I_n = torch.eye(n, dtype=torch.float64, device="cuda")
    acc = {"sigma_err": (torch.max(torch.abs(s - sig)) / sig[0]).item(),
           "residV": (torch.linalg.norm(A @ V - U * s[None, :]) / nA).item(),
           "residU": (torch.linalg.norm(A.T @ U - V * s[None, :]) / nA).item(),
           "orthU": torch.linalg.norm(U.T @ U - I_n).item(), "orthV": torch.linalg.norm(V.T @ V - I_n).item()}
    # paper-style count: the polar steps (Section 6 counts per QR- and Cholesky-based step),
    # H = U_p^T A and U = U_p V (2 m n^2 each) and 9 n^3 for the symmetric eigensolver (Table 1)
    fl = info["it_qr"] * (2 * (2 * (m + n) * n * n - 2 * n ** 3 / 3) + 2 * m * n * n) \
        + info["it_chol"] * (3 * m * n * n + n ** 3 / 3) + 4 * m * n * n + 9 * n ** 3
    t = statistics.median(ms) / 1e3
    cpu = None
    if not args.no_cpu_baseline:
        # the oracle's definition of the result (the LAPACK SVD through numpy), timed once on the host
        import oracle as O
        t0 = time.perf_counter()
        O.full.gesvd(p.A)
        cpu = {"value": 1.0 / (time.perf_counter() - t0), "unit": "solves/s", "cores": os.cpu_count(),
               "kind": "oracle", "sample": f"1 full SVD of the {m}x{n} matrix (numpy/LAPACK FP64)"}
    print(json.dumps({"workload": f"QDWH-SVD, all {n} triplets of the {m}x{n} matrix (sigma log-spaced 1..1e-12)",
                      "precision": args.precision, "ms_median": 1e3 * t, "solves_per_s": 1 / t,
                      "paper_flop_tflops": fl / t / 1e12,
                      "gemm_tflops": prof["gemm_flops"] / prof["gemm_ms"] * 1e-9 if prof["gemm_ms"] else None,
                      "gemm_share": prof["gemm_ms"] / sum(ms), "accuracy": acc,
                      "cpu_baseline": cpu,
                      "info": {k: info[k] for k in ("it_qr", "it_chol", "nodes", "leaves", "depth", "median_splits",
                                                    "jacobi_sweeps", "orthonormalized", "max_offblock")}}),
          flush=True)


def run_batched(args):
    """512 independent EIG problems (n uniform in [64, 1024], lambda ~ U[-1, 1], top 10 % each)
    through qdwhp_eig_batched; FP64 or mixed."""
    import torch

    from paper_2104_14186_gb300 import build
    build.build()
    from paper_2104_14186_gb300 import inputs as I
    from paper_2104_14186_gb300 import qdwhp as Q

    tuning = None
    if args.tune:
        # launch-shape table: reuse a saved one, else tune on this device and save it
        from paper_2104_14186_gb300 import autotune
        if os.path.exists(args.tune):
            res = autotune.load(args.tune)
        else:
            # the batched workload's sizes (64..1024) and concurrency: tune its throughput
            res = autotune.tune(classes=(0, 1, 2, 3), reps=2, objective="throughput", batch=32,
                                concurrency=args.concurrency)
            autotune.save(res, args.tune)
        autotune.apply(res)
        tuning = {"table": res["table"], "path": args.tune}
    if args.count is None:
        args.count = 512
    sizes = I.batch_sizes(args.count, 4000)
    As = [I.eig_uniform_device(int(n), 4000 + i, 0.10)[0] for i, n in enumerate(sizes)]
    prec = precision_code(Q, args.precision)
    Q.eig_batched(As[:8], 0.10, concurrency=args.concurrency, precision=prec, zolo_r=args.zolo)    # warm-up
    torch.cuda.synchronize()
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        res, sts = Q.eig_batched(As, 0.10, concurrency=args.concurrency, precision=prec, zolo_r=args.zolo)
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t0)
        assert all(s == 0 for s in sts), sts
    fl = sum(3 * (n ** 3 + n ** 3 / 3 + 2 * n ** 3) + 4 / 3 * n ** 3 for n in sizes)
    t = statistics.median(times)
    # one-at-a-time baseline: the same problems solved one after another on one stream
    sequential = None
    if args.sequential:
        o = Q.default_opts(precision=prec, zolo_r=args.zolo)
        ws = Q.workspace(max(Q.lib().qdwhp_eig_workspace_bytes(int(n), __import__("ctypes").byref(o)) for n in sizes))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for A in As:
            Q.eig(A, fraction=0.10, ws=ws, precision=prec, zolo_r=args.zolo)
        torch.cuda.synchronize()
        ts = time.perf_counter() - t0
        sequential = {"solves_per_s": args.count / ts, "ms_per_batch": 1e3 * ts,
                      "batching_gain": ts / t}
        del ws
    # accuracy of every result against the constructed spectra (outside the timed region)
    import numpy as np
    worst_lam, worst_res = 0.0, 0.0
    for i, (A, r) in enumerate(zip(As, res)):
        lam_i = np.random.default_rng(4000 + i).uniform(-1.0, 1.0, int(sizes[i]))   # the generator's spectrum
        true = torch.from_numpy(np.sort(lam_i)[::-1][: r.lam.shape[0]].copy()).to(A.device)
        worst_lam = max(worst_lam, torch.max(torch.abs(r.lam - true)).item())
        worst_res = max(worst_res, (torch.linalg.norm(A @ r.V - r.V * r.lam[None, :]) / torch.linalg.norm(A)).item())
    print(json.dumps({"workload": f"batched QDWHpartial-EIG: {args.count} matrices, n in [64, 1024], top 10 %",
                      "precision": args.precision, "zolo_r": args.zolo, "concurrency": args.concurrency,
                      "solves_per_s": args.count / t, "ms_per_batch": 1e3 * t, "alg_tflops_lower_bound": fl / t / 1e12,
                      "max_lam_err": worst_lam, "max_resid": worst_res, "tuning": tuning,
                      "one_at_a_time": sequential}), flush=True)


def serve_input(I, r):
    """One request's matrix, generated on the GPU at its arrival (butterfly orthogonal factors,
    known spectrum)."""
    if r["kind"] == "eig":
        return I.eig_butterfly_device(r["n"], r["seed"], r["fraction"])
    return I.svd_butterfly_device(r["m"], r["n"], r["seed"], r["fraction"])


def serve_once(Q, I, reqs, arrivals, prec_name, args, sample_every=40):
    """Submits every request at its arrival time (its input drawn on the GPU then), releases
    completed ones as it goes, and returns latency statistics and the sampled results."""
    import numpy as np
    import torch
    prec = precision_code(Q, prec_name)
    extra = {"precision": prec}
    svd_extra = dict(extra, refine_steps=args.refine if prec_name.startswith("mixed") else 0)
    q = Q.Queue(args.budget_gb << 30, max_slots=args.concurrency)
    inflight, lat, done_t, first_t, samples = {}, [], [], None, []

    def reap(block=False):
        for rid in list(inflight):
            st = q.poll(rid) if not block else 0
            if block:
                q.wait(rid, 3600000)
            elif st == Q.QDWHP_PENDING:
                continue
            t_sub, _, t_done = q.times(rid)
            lat.append(t_done - t_sub)
            done_t.append(t_done)
            i, A, spec, k = inflight.pop(rid)
            if i % sample_every == 0:
                res = q.wait(rid, 0)
                samples.append((i, reqs[i]["kind"], A, spec, k, res))
            q.release(rid)

    torch.cuda.synchronize()
    start = time.perf_counter()
    for i, (r, ta) in enumerate(zip(reqs, arrivals)):
        delay = start + ta - time.perf_counter()
        if delay > 0:
            time.sleep(delay)
        A, spec, k = serve_input(I, r)
        rid = q.submit_eig(A, k, **extra) if r["kind"] == "eig" else q.submit_svd(A, k, **svd_extra)
        first_t = first_t if first_t is not None else q.times(rid)[0]
        inflight[rid] = (i, A, spec, k)
        reap()
    reap(block=True)
    q.close()
    worst = {"lam_err": 0.0, "sigma_err": 0.0, "resid": 0.0, "resid_request": None}
    for i, kind, A, spec, k, res in samples:
        if kind == "eig":
            true = torch.from_numpy(np.sort(spec)[::-1][:k].copy()).to(A.device)
            worst["lam_err"] = max(worst["lam_err"], torch.max(torch.abs(res.lam - true)).item())
            rr = torch.linalg.norm(A @ res.V - res.V * res.lam[None, :]) / torch.linalg.norm(A)
        else:
            true = torch.from_numpy(spec[:k].copy()).to(A.device)
            worst["sigma_err"] = max(worst["sigma_err"], torch.max(torch.abs(res.sigma - true)).item())
            rr = max(torch.linalg.norm(A @ res.V - res.U * res.sigma[None, :]),
                     torch.linalg.norm(A.T @ res.U - res.V * res.sigma[None, :])) / torch.linalg.norm(A)
        if rr.item() > worst["resid"]:
            worst["resid"] = rr.item()
            worst["resid_request"] = dict(reqs[i], index=i, k=k)
    return {"precision": prec_name, "solves_per_s": len(lat) / (max(done_t) - first_t),
            "p50_ms": 1e3 * float(np.percentile(lat, 50)), "p99_ms": 1e3 * float(np.percentile(lat, 99)),
            "max_ms": 1e3 * float(np.max(lat)), "wall_s": max(done_t) - first_t,
            "checked": len(samples), "worst_sampled": worst}


def run_serve(args):
    """Poisson-arrival stream of mixed EIG / SVD requests through the qdwhp queue (continuous
    batching, HBM-budget admission): 2000 requests by default, EIG n in [128, 8192], SVD n in
    [128, 4096] with m in [n, 2n] and sigma log-spaced to 1e-10, fractions 1-20 %.  The arrival
    rate is 80 % of the calibrated capacity of --rate-from (its first 48 requests submitted at
    once), and every precision of --precisions sees the same arrivals.  Reports p50 / p99
    latency (completion - submission) and solves/s, and the worst error of 50 evenly spaced
    results against their known spectra.  --count takes a prefix of the 2000-request stream."""
    import numpy as np
    import torch

    from paper_2104_14186_gb300 import build
    build.build()
    from paper_2104_14186_gb300 import inputs as I
    from paper_2104_14186_gb300 import qdwhp as Q

    count = args.count if args.count is not None else 2000
    reqs, gaps = I.serving_stream(2000, 5000)
    reqs, gaps = reqs[:count], gaps[:count]      # a prefix of the 2000-request stream
    names = args.precisions.split(",") if args.precisions else [args.precision]
    rate = args.rate
    cal = None
    if rate <= 0:
        ref = args.rate_from or names[0]
        prec = precision_code(Q, ref)
        q = Q.Queue(args.budget_gb << 30, max_slots=args.concurrency)
        ncal = min(48, count)
        inputs = [serve_input(I, r) for r in reqs[:ncal]]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ids = [q.submit_eig(A, k, precision=prec) if r["kind"] == "eig" else
               q.submit_svd(A, k, precision=prec, refine_steps=args.refine if ref.startswith("mixed") else 0)
               for r, (A, _, k) in zip(reqs[:ncal], inputs)]
        for rid in ids:
            q.wait(rid, 3600000)
        cal = {"precision": ref, "requests": ncal, "capacity_per_s": ncal / (time.perf_counter() - t0)}
        q.close()
        del inputs
        rate = 0.8 * cal["capacity_per_s"]
    arrivals = np.cumsum(gaps / rate)
    results = []
    for name in names:
        results.append(serve_once(Q, I, reqs, arrivals, name, args, sample_every=max(1, count // 50)))
        print(json.dumps({"partial": True, "arrival_rate_per_s": rate, "result": results[-1]}), flush=True)
    neig = sum(1 for r in reqs if r["kind"] == "eig")
    print(json.dumps({"workload": f"serving: {count} Poisson-arrival requests ({neig} EIG n in [128, 8192], "
                                  f"{count - neig} SVD n in [128, 4096] m in [n, 2n], sigma to 1e-10), "
                                  "fractions 1-20 %, inputs drawn on the GPU at arrival",
                      "arrival_rate_per_s": rate, "calibration": cal, "concurrency": args.concurrency,
                      "budget_gb": args.budget_gb, "refine_steps_mixed_svd": args.refine, "results": results}),
          flush=True)


def run_single(args):
    """One untimed solve of the workload: the command the ncu launch-list capture runs."""
    import numpy as np
    import torch

    from paper_2104_14186_gb300 import build
    build.build()
    from paper_2104_14186_gb300 import qdwhp as Q

    p = make_problem(SEED)
    A = torch.from_numpy(np.ascontiguousarray(p.A)).cuda()
    launches0 = Q.launch_count()
    r = Q.svd(A, k=p.k, precision=precision_code(Q, args.precision))
    torch.cuda.synchronize()
    print(json.dumps({"single_solve": True, "precision": args.precision, "launches": Q.launch_count() - launches0,
                      "ell": r.info["ell"], "ms": r.info["ms_total"]}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip the emulated and mixed-emulated solves reported beside the FP64 headline")
    ap.add_argument("--precision", choices=["fp64", "mixed", "emulated", "mixed-emulated"], default="fp64")
    ap.add_argument("--refine", type=int, default=0, help="FP64 refinement steps on Q2 (SVD)")
    ap.add_argument("--tune", default=None,
                    help="batched: launch-shape table (JSON) to load, or to tune on this device and write")
    ap.add_argument("--zolo", type=int, default=0, help="Zolo-PD of order r in place of the QDWH steps (0: QDWH)")
    ap.add_argument("--kernel", choices=["gemm"], default=None,
                    help="time one building block in isolation instead of the full solve")
    ap.add_argument("--single", action="store_true", help="one untimed solve (for profiler launch lists)")
    ap.add_argument("--eig16384", action="store_true", help="time the n = 16384 clustered EIG workload")
    ap.add_argument("--batched", action="store_true", help="time the batched EIG workload")
    ap.add_argument("--gesvd", action="store_true", help="time the full-spectrum QDWH-SVD of the 4096^2 workload")
    ap.add_argument("--serve", action="store_true", help="run the serving stream")
    ap.add_argument("--count", type=int, default=None, help="batched: matrices (512); serve: requests (2000)")
    ap.add_argument("--concurrency", type=int, default=8)
    ap.add_argument("--budget-gb", type=int, default=96)
    ap.add_argument("--rate-from", default=None, help="serve: precision whose calibrated capacity sets the rate")
    ap.add_argument("--sequential", action="store_true",
                    help="batched: also time the same problems one after another on one stream")
    ap.add_argument("--rate", type=float, default=0.0)
    ap.add_argument("--fraction", type=float, default=0.01)
    ap.add_argument("--precisions", default=None,
                    help="--eig16384: comma-separated precisions to time on the same matrix")
    ap.add_argument("--cpu-baseline", action="store_true",
                    help="--eig16384: also time the FP64 oracle once on the host cores")
    args = ap.parse_args()
    if args.eig16384:
        run_eig_large(args)
        return
    if args.batched:
        run_batched(args)
        return
    if args.gesvd:
        run_gesvd(args)
        return
    if args.serve:
        run_serve(args)
        return
    if args.single:
        run_single(args)
        return
    if args.kernel == "gemm":
        run_kernel_gemm(args)
        return
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
