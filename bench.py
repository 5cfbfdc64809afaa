#!/usr/bin/env python
"""PowerURV throughput on one GB300 (or N replicas), printed as ONE JSON line.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--mode mixed|fp64|fp64emu] [--m M] [--n N] [--q Q] [--no-reorth]
                    [--workload urv|batched|adjoint|rsvd]

--mode fp64emu runs the FP64 algorithm with every product emulated on the BF16
tensor cores (8 fixed-point slices, exact sums).  --workload batched times the
batched FP32 engine (4096 matrices, n ~ U[16,256], m ~ U[n,2n], q = 2, one
persistent launch) in matrices/s; --workload adjoint times the FP64 reverse
mode (m = n = 2048, q = 2) in seconds per backward; --workload rsvd times the
randomized SVD (m = n = 8192, l = 256).
The default is the PowerURV factorization below.

A step is one full PowerURV factorization A = U R V^T (Section 3 of the
paper): Gaussian draw, q power steps with re-orthonormalisation, the QR of
Eq. (5) and the QR of Eq. (6), all on the GPU through the C ABI.  The
metric is algorithmic TFLOP/s:
    F = 2(2q+1) m n^2 + q QR(m,n) + q QR(n,n) + QR(m,n)   (reorth, q >= 1)
    F = 2(2q+1) m n^2 + QR(n,n) + QR(m,n)                 (otherwise)
    QR(r,n) = 2 (2 r n^2 - 2 n^3 / 3)   (factor + explicit Q)
counted once per product (compensated slices are not counted as extra work).

Inputs are synthetic (Section 5's recipe): A = Uh diag(sigma) Vh^T with Haar
factors, sigma_j = 10^(-6 (j-1)/(n-1)), built on the device; A (8 m n bytes)
is larger than L2, so consecutive steps do not hit in L2.

--impl reference times the FP64 CPU oracle (the only reference this project
has: the paper ships no code) on the host cores, on a bounded sample of the
same workload, and prints the same metric.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = ("PowerURV sec & TFLOP/s, n=16384 q=2: mixed vs FP64 at "
          "‖A−URV*‖/‖A‖≤1e-6")


def qr_flops(r: int, n: int) -> float:
    return 2.0 * (2.0 * r * n * n - 2.0 * n ** 3 / 3.0)


def urv_flops(m: int, n: int, q: int, reorth: bool) -> float:
    f = 2.0 * (2 * q + 1) * m * n * n
    if reorth and q >= 1:
        return f + q * qr_flops(m, n) + q * qr_flops(n, n) + qr_flops(m, n)
    return f + qr_flops(n, n) + qr_flops(m, n)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--mode", choices=["mixed", "mixed16", "fp32", "fp64", "fp64emu"], default="mixed",
                    help="mixed: BF16 power steps; mixed16: FP16 power steps; fp32: 4 exact slices; fp64; "
                         "fp64emu.  --workload adjoint: fp32 (the default there), fp64 or fp64emu")
    ap.add_argument("--m", type=int, default=0, help="rows (default n)")
    ap.add_argument("--n", type=int, default=16384)
    ap.add_argument("--q", type=int, default=2)
    ap.add_argument("--no-reorth", action="store_true")
    ap.add_argument("--cpu-sample-n", type=int, default=2560,
                    help="size of the oracle's bounded CPU sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-profile", action="store_true", help="skip per-kernel event timing")
    ap.add_argument("--workload", choices=["urv", "batched", "adjoint", "rsvd", "product"], default="urv")
    ap.add_argument("--engine", choices=["f64", "tc", "tcx"], default="tcx",
                    help="product: FP64 DFMA engine, plain BF16 slices (tc), or exact slices (tcx)")
    ap.add_argument("--slices", type=int, default=4, help="product: slices per operand")
    ap.add_argument("--k", type=int, default=0, help="product: reduction length (default n)")
    ap.add_argument("--update", action="store_true", help="product: C = C - A B instead of C = A B")
    ap.add_argument("--matrix", choices=["haar", "gaussian"], default="haar",
                    help="urv: Haar-factor matrix with sigma_j = 10^(-6(j-1)/(n-1)), or Gaussian entries")
    ap.add_argument("--rank", type=int, default=256, help="rsvd: target rank l")
    ap.add_argument("--count", type=int, default=4096, help="batched: number of matrices")
    ap.add_argument("--variant", type=int, default=-1, help="batched: kernel variant (-1 = autotune)")
    ap.add_argument("--fp64-n", type=int, default=-1,
                    help="size of the native FP64 comparison run (-1 = the bench's n, 0 = skip; "
                         "about 94 s at n=16384)")
    ap.add_argument("--fp64emu-n", type=int, default=-1,
                    help="mixed mode: size of the FP64-emulation comparison run (-1 = the bench's n, 0 = skip)")
    a = ap.parse_args()
    a.m = a.m or a.n
    a.reorth = not a.no_reorth
    if a.fp64_n < 0:
        a.fp64_n = a.n
    if a.fp64emu_n < 0:
        a.fp64emu_n = a.n
    return a


# ------------------------------------------------------------------ clocks --
class ClockSampler:
    """nvidia-smi samples (200 ms) of SM clock and throttle reasons while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.out = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-i", str(self.dev), "-lms", "200"], stdout=self.out, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.out.close()

    def summary(self):
        if self.proc is None or not self.path:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------ cpu oracle ---
def cpu_oracle_run(n: int, q: int, reorth: bool, reps: int = 1):
    """Time the FP64 CPU oracle (as it stands) on an n x n sample; returns (TFLOP/s, seconds, cores)."""
    import numpy as np
    import oracle
    from paper_1812_06007_gb300 import workloads as W
    oracle.build()
    A = W.test_matrix_np(n, n, W.sigma_profile("exponential", n, decades=6))
    times = []
    for _ in range(reps):
        t0 = time.perf_counter()
        oracle.urv(A, q, reorth, W.SEED_G)
        times.append(time.perf_counter() - t0)
    t = min(times)
    cores = int(os.environ.get("OMP_NUM_THREADS", 0)) or os.cpu_count()
    return urv_flops(n, n, q, reorth) / t / 1e12, t, cores


def run_reference(a):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    n = a.cpu_sample_n
    for _ in range(a.warmup):
        cpu_oracle_run(n, a.q, a.reorth)
    vals, secs = [], []
    cores = os.cpu_count()
    for _ in range(a.steps):
        v, t, cores = cpu_oracle_run(n, a.q, a.reorth)
        vals.append(v)
        secs.append(t)
    value = statistics.median(vals)
    sample = f"PowerURV m=n={n} q={a.q} reorth={int(a.reorth)} (FP64 C oracle, OpenMP), one factorization per step"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": a.gpus,
        "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1e3 * statistics.median(secs),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": f"PowerURV m=n={a.n} q={a.q} reorth={int(a.reorth)} ({a.mode}); "
                               f"CPU sample m=n={n}", "m": a.m, "n": a.n, "q": a.q, "reorth": a.reorth,
                   "mode": a.mode, "l2": "n/a (CPU)"},
        "cpu_baseline": {"value": value, "unit": "TFLOP/s", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- ours -----
def max_over_ranks(value: float, device=None) -> float:
    """Max of a per-rank timing over the process group (a plain host value when not distributed)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device if device is not None else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_value(flops_per_step: float, world: int, ms_step_max: float) -> float:
    """Whole-job TFLOP/s of N independent replicas (weak scaling): all ranks' work over the slowest rank."""
    return flops_per_step * world / (ms_step_max * 1e-3) / 1e12


def run_ours(a):
    import torch
    import torch.distributed as dist

    from paper_1812_06007_gb300 import binding as B
    from paper_1812_06007_gb300 import build as Bld
    from paper_1812_06007_gb300 import workloads as W

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", torch.cuda.current_device())
    Bld.build()
    B.lib()
    mode = {"mixed": B.PURL_MODE_MIXED_BF16, "mixed16": B.PURL_MODE_MIXED_FP16, "fp32": B.PURL_MODE_FP32,
            "fp64": B.PURL_MODE_FP64, "fp64emu": B.PURL_MODE_FP64_EMU}[a.mode]
    m, n, q, reorth = a.m, a.n, a.q, a.reorth

    if a.matrix == "gaussian":
        A = W.gaussian_matrix_torch(m, n, 2024 + rank, device=dev)
    else:
        A = W.test_matrix_torch(m, n, W.sigma_profile("exponential", n, decades=6), device=dev)
    U = B.empty_colmajor(m, n, dev)
    R = B.empty_colmajor(n, n, dev)
    V = B.empty_colmajor(n, n, dev)
    ws = torch.empty(B.purl_urv_workspace_bytes(m, n, mode), dtype=torch.uint8, device=dev)
    seed = W.SEED_G + rank
    stream = torch.cuda.current_stream()

    def step():
        B.purl_urv_factor(A, q, reorth, seed, mode=mode, out=(U, R, V), workspace=ws, stream=stream)

    for _ in range(a.warmup):
        step()
    torch.cuda.synchronize()
    if B.purl_device_status() != B.PURL_OK:
        raise RuntimeError("device status not ok after warm-up")

    # ---- timed region (device resident) ----
    if not a.no_profile:
        # per-kernel CUDA events inside the timed region, on every 8th launch of
        # each kernel (after its first 8): enough for per-kernel averages while
        # keeping the event records from stretching the step
        B.purl_profile_reset()
        B.purl_profile_set_stride(8)
        B.purl_profile_enable(True)
    launches0 = B.purl_launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(dev.index) as clk:
        e0.record(stream)
        for _ in range(a.steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    launches = B.purl_launch_count() - launches0
    ms_total = e0.elapsed_time(e1)
    prof = B.purl_profile_read() if not a.no_profile else None
    prof_named = B.purl_profile_read_named() if not a.no_profile else None
    B.purl_profile_enable(False)
    ms_total = max_over_ranks(ms_total, dev)
    ms_step = ms_total / a.steps
    flops = urv_flops(m, n, q, reorth)
    value = replica_value(flops, world, ms_step)

    # ---- errors of the last factorization (random-probe estimators, FP64) ----
    errs = probe_errors(A, U, R, V)

    # ---- end to end: host A -> device, factor, U R V -> host ----
    e2e = None
    if not a.no_e2e:
        e2e = end_to_end(a, A, U, R, V, ws, mode, seed, world, dev, B)

    # ---- the FP64 path on the same recipe (the "vs FP64" of the metric) ----
    fp64 = fp64emu = None
    if a.mode in ("mixed", "mixed16", "fp32", "fp64emu") and (a.fp64_n > 0 or a.fp64emu_n > 0):
        del ws
        torch.cuda.empty_cache()
    if a.mode in ("mixed", "mixed16", "fp32", "fp64emu") and a.fp64_n > 0:
        fp64 = fp64_compare(a, dev, B, W, seed, B.PURL_MODE_FP64, a.fp64_n, A)
    if a.mode in ("mixed", "mixed16", "fp32") and a.fp64emu_n > 0:
        fp64emu = fp64_compare(a, dev, B, W, seed, B.PURL_MODE_FP64_EMU, a.fp64emu_n, A)

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return 0

    # ---- roofline of the dominant kernel function ----
    clocks = clk.summary()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    roof = roofline(prof, prof_named, a.steps, a.mode, sm_mhz=clocks.get("sm_mhz"), sms=sms)
    if roof is not None and prof_named:
        roof["share_of_step"] = by_function(prof_named)[roof["kernel"]]["ms"] / a.steps / ms_step
        attach_traffic(roof)
    cpu = None
    if not a.no_cpu_baseline and world == 1:
        v, t, cores = cpu_oracle_run(a.cpu_sample_n, q, reorth)
        cpu = {"value": v, "unit": "TFLOP/s", "cores": cores, "kind": "oracle",
               "sample": f"PowerURV m=n={a.cpu_sample_n} q={q} reorth={int(reorth)}, FP64 C oracle "
                         f"(OpenMP), one factorization, {t:.2f} s"}
    # The stdout line stays short (the accuracy gate of the metric and the FP64 comparison come
    # before anything long); the per-kernel breakdown goes to stderr as a second JSON object.
    acc = {"recon_rel_fro": errs["recon_rel_fro"], "orth_U_fro": errs["orth_U_fro"],
           "orth_V_fro": errs["orth_V_fro"], "meets_1e-6": errs["recon_rel_fro"] <= 1e-6}
    line = {
        "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "data": "synthetic",
        "dtype": {"mixed": "bf16+f64", "mixed16": "fp16+bf16+f64", "fp32": "f32 (4 bf16 slices, exact sums)",
                  "fp64": "f64", "fp64emu": "f64 (emulated: 8 bf16 slices, exact sums)"}[a.mode],
        "config": {"workload": f"PowerURV m={m} n={n} q={q} reorth={int(reorth)} {a.mode}",
                   "m": m, "n": n, "q": q, "reorth": reorth, "mode": a.mode,
                   "matrix": ("Gaussian entries" if a.matrix == "gaussian"
                              else "Haar factors, sigma 10^(-6(j-1)/(n-1))"), "parallelism": f"replicas{world}",
                   "l2": f"inputs larger than L2 (A is {8 * m * n / 2**30:.1f} GiB)"},
        "sec_per_factorization": ms_step * 1e-3,
        "accuracy": acc,
        "fp64_path": fp64,
        "speedup_vs_fp64_path": ((fp64["sec"] / (ms_step * 1e-3)) if (fp64["m"], fp64["n"]) == (m, n)
                                 else value / fp64["tflops"]) if fp64 else None,
        "fp64emu_path": fp64emu,
        "flops_per_step": flops,
        "gpu_launches": int(launches),
        "clocks": clocks,
        "roofline": roof,
        "cpu_baseline": cpu,
        "e2e": e2e,
    }
    print(json.dumps(line), flush=True)
    if prof_named:
        funcs = by_function(prof_named)
        detail = {"kernel_classes": prof,
                  "kernel_functions_ms_per_step": {k: round(v["ms"] / a.steps, 3) for k, v in
                                                   sorted(funcs.items(), key=lambda kv: -kv[1]["ms"])},
                  "labels": {k: {"launches": v["launches"], "ms_per_step": v["ms"] / a.steps,
                                 "tflops": v["flops"] / max(v["ms"], 1e-9) / 1e9}
                             for k, v in sorted(prof_named.items(), key=lambda kv: -kv[1]["ms"])}}
        print("per-kernel " + json.dumps(detail), file=sys.stderr, flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def fp64_compare(a, dev, B, W, seed, mode, n, A_main=None):
    """Time an FP64-accurate mode (native FP64, or FP64 emulated on the tensor cores) at size n on the
    same recipe: one factorization at n = 1024 first (kernel attributes, allocator), then one timed
    factorization at n with CUDA events, and its probe errors."""
    import torch
    m = n if a.m == a.n else int(round(a.m * n / a.n))
    stream = torch.cuda.current_stream()
    w = min(n, 1024)
    Aw = W.gaussian_matrix_torch(w, w, 99, device=dev)
    B.purl_urv_factor(Aw, a.q, a.reorth, seed, mode=mode, stream=stream)
    torch.cuda.synchronize()
    del Aw
    if A_main is not None and tuple(A_main.shape) == (m, n) and a.matrix == "haar":
        A = A_main  # the same matrix the timed steps factored
    else:
        A = W.test_matrix_torch(m, n, W.sigma_profile("exponential", n, decades=6), device=dev)
    U, R, V = B.empty_colmajor(m, n, dev), B.empty_colmajor(n, n, dev), B.empty_colmajor(n, n, dev)
    ws = torch.empty(B.purl_urv_workspace_bytes(m, n, mode), dtype=torch.uint8, device=dev)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    B.purl_urv_factor(A, a.q, a.reorth, seed, mode=mode, out=(U, R, V), workspace=ws, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    if B.purl_device_status() != B.PURL_OK:
        raise RuntimeError("device status not ok after the FP64 comparison run")
    sec = e0.elapsed_time(e1) * 1e-3
    errs = probe_errors(A, U, R, V)
    del ws, A, U, R, V
    torch.cuda.empty_cache()
    return {"m": m, "n": n, "q": a.q, "reorth": a.reorth, "sec": sec,
            "tflops": urv_flops(m, n, a.q, a.reorth) / sec / 1e12,
            "recon_rel_fro": errs["recon_rel_fro"], "orth_U_fro": errs["orth_U_fro"],
            "orth_V_fro": errs["orth_V_fro"], "timed": "1 factorization (after one at n=1024)"}


def probe_errors(A, U, R, V, k: int = 16):
    """||A - U R V^T||_F / ||A||_F and ||I - U^T U||_F, ||I - V^T V||_F / sqrt(n), estimated
    with k Gaussian probe vectors (E ||M X||_F^2 = k ||M||_F^2)."""
    import torch
    m, n = A.shape
    g = torch.Generator(device=A.device)
    g.manual_seed(12345)
    X = torch.randn(n, k, generator=g, device=A.device, dtype=torch.float64)
    AX = A @ X
    E = AX - U @ (R @ (V.t() @ X))
    recon = (torch.linalg.norm(E) / torch.linalg.norm(AX)).item()
    ou = (torch.linalg.norm(U.t() @ (U @ X) - X) / math.sqrt(k)).item()
    ov = (torch.linalg.norm(V.t() @ (V @ X) - X) / math.sqrt(k)).item()
    return {"recon_rel_fro": recon, "orth_U_fro": ou, "orth_V_fro": ov, "estimator": f"{k} Gaussian probes"}


def end_to_end(a, A, U, R, V, ws, mode, seed, world, dev, B):
    """Same factorization through the public API with host memory on both ends: every step copies A
    from pinned host memory to the device and U, R, V back.  Host-to-device and device-to-host
    copies run on two streams of their own and device buffers are doubled, so step i+1's input copy
    and step i-1's output copies overlap step i's factorization; the timed region runs from the
    first H2D copy to the last D2H copy.  The copies' own durations are reported beside it."""
    import torch
    m, n = A.shape
    hA = torch.empty((n, m), dtype=torch.float64, pin_memory=True).t()
    hA.copy_(A)
    hU = torch.empty((n, m), dtype=torch.float64, pin_memory=True).t()
    hR = torch.empty((n, n), dtype=torch.float64, pin_memory=True).t()
    hV = torch.empty((n, n), dtype=torch.float64, pin_memory=True).t()
    dA = [B.empty_colmajor(m, n, dev) for _ in range(2)]
    outs = [(U, R, V), (B.empty_colmajor(m, n, dev), B.empty_colmajor(n, n, dev), B.empty_colmajor(n, n, dev))]
    comp = torch.cuda.current_stream()
    h2d, d2h = torch.cuda.Stream(device=dev), torch.cuda.Stream(device=dev)
    ev = lambda: torch.cuda.Event()
    tev = lambda: torch.cuda.Event(enable_timing=True)
    a_ready, a_free = [ev(), ev()], [ev(), ev()]
    done, out_free = [ev(), ev()], [ev(), ev()]
    for e in a_free + out_free:
        e.record(comp)
    marks = {}

    def load(i):
        b = i % 2
        mk = marks.setdefault(i, [tev() for _ in range(4)])
        with torch.cuda.stream(h2d):
            h2d.wait_event(a_free[b])
            mk[0].record(h2d)
            # column-major m x n is a contiguous n x m row-major array: copying the
            # contiguous bases makes each copy one straight DMA of pinned memory
            dA[b].t().copy_(hA.t(), non_blocking=True)
            mk[1].record(h2d)
            a_ready[b].record(h2d)

    def factor_and_store(i):
        b = i % 2
        mk = marks[i]
        comp.wait_event(a_ready[b])
        comp.wait_event(out_free[b])
        Ub, Rb, Vb = outs[b]
        B.purl_urv_factor(dA[b], a.q, a.reorth, seed, mode=mode, out=(Ub, Rb, Vb), workspace=ws, stream=comp)
        done[b].record(comp)
        a_free[b].record(comp)
        with torch.cuda.stream(d2h):
            d2h.wait_event(done[b])
            mk[2].record(d2h)
            hU.t().copy_(Ub.t(), non_blocking=True)
            hR.t().copy_(Rb.t(), non_blocking=True)
            hV.t().copy_(Vb.t(), non_blocking=True)
            mk[3].record(d2h)
            out_free[b].record(d2h)

    load(0)
    factor_and_store(0)
    torch.cuda.synchronize()
    marks.clear()
    steps = max(1, min(a.steps, 3))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(comp)
    h2d.wait_event(e0)
    load(0)
    for i in range(steps):
        # the next step's input copy is queued before this step's kernels, so it runs beside them
        if i + 1 < steps:
            load(i + 1)
        factor_and_store(i)
    comp.wait_stream(d2h)
    e1.record(comp)
    torch.cuda.synchronize()
    ms = max_over_ranks(e0.elapsed_time(e1) / steps, dev)
    h2d_ms = sum(mk[0].elapsed_time(mk[1]) for mk in marks.values()) / steps
    d2h_ms = sum(mk[2].elapsed_time(mk[3]) for mk in marks.values()) / steps
    bi, bo = 8 * m * n, 8 * (m * n + 2 * n * n)
    return {"value": urv_flops(m, n, a.q, a.reorth) * world / (ms * 1e-3) / 1e12, "unit": "TFLOP/s",
            "ms_per_step": ms, "h2d_bytes_per_step": bi, "d2h_bytes_per_step": bo,
            "h2d_ms": h2d_ms, "d2h_ms": d2h_ms,
            "h2d_gbs": bi / (h2d_ms * 1e-3) / 1e9, "d2h_gbs": bo / (d2h_ms * 1e-3) / 1e9,
            "steps": steps,
            "pipelined": "H2D and D2H copies on two streams of their own, double-buffered device inputs and outputs"}


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) per launch of a kernel function, averaged
# over every launch of one ncu capture of the bench's own step (summary and command under profiles/).
# It is reported only while the source that determines the kernel's traffic -- its configuration, the
# kernel, its launch and the tile dispatch, as regions of its source file -- still has the hash it had
# when captured.
TRAFFIC = {
    # 5906 launches of one mixed n = 16384 factorization: 770.37 GB read + 235.18 GB written
    "tcx_gemm_kernel": {
        "src": "paper_1812_06007_gb300/csrc/gemm_tcx.cu",
        "regions": [("template <int S, bool ALL, int BN>\nstruct TcxCfg {",
                     "template <int S>\n__global__ void __launch_bounds__(256) split_exact_kernel("),
                    ("template <int S, bool ALL, int BN>\nint launch_tcx(", "}  // namespace\n"),
                    ("int tcx_gemm_view_impl(", "int tcx_gemm_view(")],
        "sha16": "4a8910c1a36b76ea",
        "bytes_per_launch": 170.26e6,
        "profile": "profiles/ncu_tcx_gemm_kernel_traffic_mixed_n16384.md"},
}


def _region_sha16(path: str, regions) -> str:
    """sha256 (16 hex digits) of the concatenated text regions [start, end) of a source file, each
    from the first occurrence of its start marker (after the previous region) to its end marker."""
    import hashlib
    with open(path, encoding="utf-8") as f:
        text = f.read()
    h = hashlib.sha256()
    for start, end in regions:
        a = text.index(start)
        b = text.index(end, a + len(start))
        h.update(text[a:b].encode("utf-8"))
    return h.hexdigest()[:16]


def attach_traffic(roof):
    t = TRAFFIC.get(roof.get("kernel"))
    if not t:
        return
    try:
        same = _region_sha16(os.path.join(ROOT, t["src"]), t["regions"]) == t["sha16"]
    except (OSError, ValueError):
        same = False
    if same:
        roof["traffic"] = t["bytes_per_launch"]
        roof["traffic_source"] = t["profile"]
    else:
        roof["traffic_note"] = f"{t['src']} changed since the ncu capture ({t['profile']})"


def fp64_peak_tflops(sm_mhz: float | None, sms: int = 152) -> float:
    """FP64 DFMA peak from the unit count and the SM clock sampled under load: 2 DFMA per clock per SM
    (4 flops), i.e. 1.26 TFLOP/s for 152 SMs at the 2070 MHz maximum (nominal GB300 FP64: 1.25)."""
    return sms * 4.0 * (sm_mhz or 2070.0) * 1e6 / 1e12


def kernel_function(label: str) -> str:
    """The CUDA kernel function a profiler label belongs to.  The tensor-core engines book their
    launches under call-site tags ("tcx outer update", "tcx emu A Y", "tc noalloc", ...), which
    name their kernel by prefix; every other label is the kernel's own name."""
    if label.startswith("tcx"):
        return "tcx_gemm_kernel"
    if label == "tc_gemm_kernel" or label.startswith("tc "):
        return "tc_gemm_kernel"
    return label


def by_function(named):
    """Per-label totals summed per kernel function; each function keeps its call sites."""
    out = {}
    for label, st in (named or {}).items():
        agg = out.setdefault(kernel_function(label),
                             {"launches": 0, "ms": 0.0, "flops": 0.0, "bytes": 0.0, "sites": {}})
        for k in ("launches", "ms", "flops", "bytes"):
            agg[k] += st[k]
        agg["sites"][label] = st
    return out


def roofline(prof, named, steps, mode, sm_mhz=None, sms=152):
    """Roofline of the dominant kernel function (by device time in the timed region).

    Call-site labels are summed per kernel function first.  Tensor-core kernels: issued BF16 flops
    (2 m n k per slice pair) over their event-timed duration against the measured sustained BF16
    peak; FP64 DFMA kernels: FP64 flops against the DFMA peak at the sampled SM clock; everything
    else: algorithmic bytes against the measured copy bandwidth."""
    funcs = by_function(named)
    if not funcs:
        return None
    peaks, src = _peaks()
    name = max(funcs, key=lambda k: funcs[k]["ms"])
    st = funcs[name]
    if st["launches"] == 0 or st["ms"] <= 0:
        return None
    sec = st["ms"] * 1e-3
    base = {"kernel": name, "launches_per_step": st["launches"] / steps,
            "avg_launch_ms": st["ms"] / st["launches"], "traffic": None,
            "share_of_step": None, "hbm_gbs_algorithmic": st["bytes"] / sec / 1e9}
    if len(st["sites"]) > 1:
        base["call_sites_ms_per_step"] = {k: round(v["ms"] / steps, 2) for k, v in
                                          sorted(st["sites"].items(), key=lambda kv: -kv[1]["ms"])[:8]}
    if name in ("tcx_gemm_kernel", "tc_gemm_kernel"):
        achieved = st["flops"] / sec / 1e12
        peak = peaks.get("bf16_tflops_sustained", 1700.0)
        base.update({"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "peak_source": f"{src} bf16 sustained (cuBLAS)",
                     "flops_counted": "issued: 2 m n k per BF16 slice pair"})
        return base
    if name == "panel_kernel" and mode in ("mixed", "mixed16", "fp32"):
        # the tensor-core QR's panel at up to 4 slices computes in FP32 (its reflector
        # parameters in FP64, its Gram matrix in integers)
        achieved = st["flops"] / sec / 1e12
        peak = FP32_LANES * 2 * (sm_mhz or 1920.0) * 1e6 / 1e12 * sms / 152
        base.update({"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak,
                     "peak_source": f"FP32 FFMA: {sms} SMs x 128 lanes x 2 flops x "
                                    f"{(sm_mhz or 1920.0):.0f} MHz (sampled SM clock)"})
        return base
    if name in ("panel_kernel", "gemm_f64_kernel", "gram_kernel") or name.startswith("gemm_f64"):
        achieved = st["flops"] / sec / 1e12
        peak = fp64_peak_tflops(sm_mhz, sms)
        base.update({"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak,
                     "peak_source": f"FP64 DFMA: {sms} SMs x 2 DFMA/clk x 2 flops x "
                                    f"{(sm_mhz or 2070.0):.0f} MHz (sampled SM clock)"})
        return base
    achieved = st["bytes"] / sec / 1e9
    peak = peaks.get("hbm_gbs", 6800.0)
    base.update({"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                 "peak_source": f"{src} hbm copy"})
    return base


# ------------------------------------------------------------- batched -----
BATCHED_METRIC = "batched PowerURV FP32 matrices/s (4096 matrices, n~U[16,256], m~U[n,2n], q=2)"
# FP32 FFMA peak: 152 SMs x 128 FP32 lanes x 2 flops per clock at the SM clock
# sampled under load (1920 MHz if no sample).
FP32_LANES = 152 * 128


def _batched_inputs(count, ms, ns):
    """Packed host FP32 A of the batched workload, built in a spawn pool (numpy QR per matrix)."""
    import concurrent.futures as cf
    import multiprocessing as mp
    import numpy as np
    from paper_1812_06007_gb300 import workloads as W
    jobs = [(int(ms[i]), int(ns[i]), i) for i in range(count)]
    workers = max(1, min(16, os.cpu_count() or 1))
    # one BLAS thread per worker: the spawned processes inherit this environment
    keys = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")
    saved = {k: os.environ.get(k) for k in keys}
    for k in keys:
        os.environ[k] = "1"
    try:
        with cf.ProcessPoolExecutor(workers, mp_context=mp.get_context("spawn")) as ex:
            mats = list(ex.map(_batched_one, jobs, chunksize=64))
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    return mats


def _batched_one(job):
    from paper_1812_06007_gb300 import workloads as W
    m, n, i = job
    return W.batched_matrix_np(m, n, i)


def run_batched(a):
    import numpy as np
    import torch
    import torch.distributed as dist
    from paper_1812_06007_gb300 import binding as B
    from paper_1812_06007_gb300 import build as Bld
    from paper_1812_06007_gb300 import workloads as W
    from paper_1812_06007_gb300.batched import Batch, flops as batch_flops

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    count, q, reorth = a.count, a.q, a.reorth
    ms, ns = W.batched_shapes(count)
    # weak scaling: every rank factors its own batch of `count` matrices (seeds offset by rank)
    mats = _batched_inputs(count, ms, ns)   # spawn pool before any GPU call
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", torch.cuda.current_device())
    Bld.build()
    B.lib()
    b = Batch(ms, ns, [W.batched_seed(i) + rank * count for i in range(count)], device=dev)
    host = b.pack_host(mats)
    b.load_packed_a(host)
    stream = torch.cuda.current_stream()
    if a.variant >= 0:
        variant, tune_ms = a.variant, None
    else:
        variant, tune_ms = b.autotune(q, reorth, stream=stream)
    for _ in range(a.warmup):
        b.factor(q, reorth, variant=variant, stream=stream)
    torch.cuda.synchronize()
    if b.status() != 0:
        raise RuntimeError("batched status not ok after warm-up")
    # the step as a CUDA graph (reset + persistent kernel), replayed K times
    gs = torch.cuda.Stream(device=dev)
    gs.wait_stream(stream)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(gs):
        b.factor(q, reorth, variant=variant, stream=gs)
        torch.cuda.synchronize()
        with torch.cuda.graph(g, stream=gs):
            b.factor(q, reorth, variant=variant, stream=gs)
    torch.cuda.synchronize()
    launches0 = B.purl_launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(dev.index) as clk, torch.cuda.stream(gs):
        e0.record(gs)
        for _ in range(a.steps):
            g.replay()
        e1.record(gs)
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    launches = 2 * a.steps  # each replay runs the graph's two kernels (counted at capture)
    assert B.purl_launch_count() == launches0
    ms_step = max_over_ranks(e0.elapsed_time(e1) / a.steps, dev)
    value = count * world / (ms_step * 1e-3)
    F = batch_flops(ms, ns, q, reorth)
    # per-matrix launches of the same device code (the baseline the single launch
    # replaces), timed on every 16th descriptor and scaled by its share of the m n^2 work
    ws = b.ensure_workspace(-1)
    torch.cuda.synchronize()
    sample = list(range(0, b.count, 16))
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    p0.record(stream)
    for d in sample:
        B.purl_urv_factor_batched(b.item_view(d), 1, b.max_m, b.max_n, q, reorth, ws, variant=variant,
                                  stream=stream)
    p1.record(stream)
    torch.cuda.synchronize()
    work = (ms * ns * ns).astype(np.float64)[b.order]
    per_matrix_ms = p0.elapsed_time(p1) * work.sum() / work[sample].sum()
    # uncaptured launches of the persistent kernel (no graph)
    u0, u1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    u0.record(stream)
    for _ in range(a.steps):
        b.factor(q, reorth, variant=variant, stream=stream)
    u1.record(stream)
    torch.cuda.synchronize()
    nograph_ms = u0.elapsed_time(u1) / a.steps
    # end to end: packed A host -> device, factor, U R V device -> host, every step
    hA = torch.from_numpy(host).pin_memory()
    hU = torch.empty(b.U.numel(), dtype=torch.float32).pin_memory()
    hR = torch.empty(b.R.numel(), dtype=torch.float32).pin_memory()
    hV = torch.empty(b.V.numel(), dtype=torch.float32).pin_memory()
    x0, x1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    x0.record(stream)
    e2e_steps = max(1, min(a.steps, 3))
    for _ in range(e2e_steps):
        b.A.copy_(hA, non_blocking=True)
        b.factor(q, reorth, variant=variant, stream=stream)
        hU.copy_(b.U, non_blocking=True)
        hR.copy_(b.R, non_blocking=True)
        hV.copy_(b.V, non_blocking=True)
    x1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(x0.elapsed_time(x1) / e2e_steps, dev)
    if b.status() != 0:
        raise RuntimeError("batched status not ok")
    # errors on a sample (FP64 products on the device)
    worst_rec = 0.0
    for i in list(range(0, count, max(1, count // 64))):
        A_ = b.a(i).double()
        worst_rec = max(worst_rec, float(torch.linalg.matrix_norm(A_ - b.u(i).double() @ b.r(i).double()
                                                                   @ b.v(i).double().t())
                                         / torch.linalg.matrix_norm(A_)))
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return 0
    csum = clk.summary()
    mhz = csum.get("sm_mhz") or 1920.0
    fp32_peak = FP32_LANES * 2 * mhz * 1e6 / 1e12
    achieved = F / (ms_step * 1e-3) / 1e12
    roof = {"bound": "alu", "kernel": "urv_batched_kernel", "achieved": achieved, "peak": fp32_peak,
            "unit": "TFLOP/s", "frac": achieved / fp32_peak, "traffic": None,
            "peak_source": f"FP32 FFMA: 152 SMs x 128 lanes x 2 flops x {mhz:.0f} MHz (sampled SM clock)",
            "flops_counted": "algorithmic PowerURV flops of every matrix (explicit Q counted)",
            "launches_per_step": 2, "avg_launch_ms": ms_step}
    cpu = None
    if not a.no_cpu_baseline and world == 1:
        cpu = _batched_cpu(mats, ms, ns, q, reorth)
    line = {
        "metric": BATCHED_METRIC, "value": value, "unit": "matrices/s", "n_gpus": world, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"batched PowerURV, {count} matrices, n~U[16,256], m~U[n,2n], q={q} "
                               f"reorth={int(reorth)}, FP32", "count": count, "q": q, "reorth": reorth,
                   "sigma": "10^(-6(j-1)/(n-1)), Haar factors", "parallelism": f"replicas{world}",
                   "l2": f"inputs larger than L2 (A is {4 * float((ms * ns).sum()) / 2**20:.0f} MiB)",
                   "variant": variant, "autotune_ms": tune_ms},
        "tflops": achieved, "flops_per_step": F,
        "per_matrix_launches": {"ms": per_matrix_ms, "matrices_per_s": count / (per_matrix_ms * 1e-3),
                                "note": "same device code, one launch per matrix, one stream; timed on every "
                                        "16th matrix (largest first) and scaled by its share of the m n^2 work"},
        "speedup_vs_per_matrix_launches": per_matrix_ms / ms_step,
        "no_graph_ms_per_step": nograph_ms,
        "errors": {"recon_rel_fro_max_sample": worst_rec, "sample": "every 64th matrix"},
        "roofline": roof, "cpu_baseline": cpu,
        "e2e": {"value": count * world / (e2e_ms * 1e-3), "unit": "matrices/s", "ms_per_step": e2e_ms,
                "h2d_bytes_per_step": 4 * b.A.numel(),
                "d2h_bytes_per_step": 4 * (b.U.numel() + b.R.numel() + b.V.numel()), "steps": e2e_steps},
        "gpu_launches": launches, "clocks": csum,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def _batched_cpu(mats, ms, ns, q, reorth, budget_s: float = 15.0):
    """The FP64 oracle on the batch's matrices in order until ~budget_s of CPU time: matrices/s."""
    import numpy as np
    import oracle
    from paper_1812_06007_gb300 import workloads as W
    oracle.build()
    done, t0 = 0, time.perf_counter()
    for i, X in enumerate(mats):
        oracle.urv(np.asarray(X, dtype=np.float64), q, reorth, W.batched_seed(i))
        done += 1
        if time.perf_counter() - t0 > budget_s:
            break
    t = time.perf_counter() - t0
    frac = float((ms[:done] * ns[:done] ** 2).sum() / (ms * ns ** 2).sum())
    # scale to the whole batch by its share of m n^2 work: matrices/s of the full mix
    return {"value": len(mats) / (t / max(frac, 1e-12)), "unit": "matrices/s",
            "cores": int(os.environ.get("OMP_NUM_THREADS", 0)) or os.cpu_count(), "kind": "oracle",
            "sample": f"first {done} matrices of the batch ({100 * frac:.1f}% of its m n^2 work) in {t:.1f} s, "
                      "FP64 C oracle (OpenMP), scaled to the full batch by work share"}


def run_batched_reference(a):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from paper_1812_06007_gb300 import workloads as W
    ms, ns = W.batched_shapes(a.count)
    mats = [W.batched_matrix_np(int(ms[i]), int(ns[i]), i) for i in range(min(a.count, 400))]
    vals = []
    cpu = None
    for _ in range(a.warmup + a.steps):
        cpu = _batched_cpu(mats, ms[:len(mats)], ns[:len(mats)], a.q, a.reorth, budget_s=10.0)
        vals.append(cpu["value"])
    vals = vals[a.warmup:]
    value = statistics.median(vals)
    cpu["value"] = value
    line = {"impl": "reference", "metric": BATCHED_METRIC, "value": value, "unit": "matrices/s",
            "n_gpus": a.gpus, "steps": a.steps, "warmup": a.warmup, "ms_per_step": a.count / value * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": f"batched PowerURV, {a.count} matrices, q={a.q}",
                                            "l2": "n/a (CPU)"},
            "cpu_baseline": cpu, "e2e": {"value": value, "unit": "matrices/s", "h2d_bytes_per_step": 0,
                                         "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------- adjoint -----
ADJOINT_METRIC = "PowerURV adjoint (reverse mode, G fixed) seconds per backward, m=n=2048 q=2 reorth"


def adjoint_flops(m, n, q, reorth):
    """Flops of the reverse call: the recomputed forward pass plus, per QR, its reverse rule
    (two n x n x m products, one m x n x n product, the triangular inverse n^3/3 and
    X R^-T, m n^2) and per power product two transposed products."""
    fwd = urv_flops(m, n, q, reorth)
    nqr_m = (q if reorth else 0) + 1
    nqr_n = (q - 1 if (reorth and q > 0) else 0) + 1
    qrb = lambda r: 2 * (2.0 * n * n * r) + 2.0 * r * n * n + n ** 3 / 3.0 + 2.0 * r * n * n
    return fwd + nqr_m * qrb(m) + nqr_n * qrb(n) + 2 * q * 2 * (2.0 * m * n * n) + 2 * (2.0 * m * n * n)


def run_adjoint(a):
    import numpy as np
    import torch
    from paper_1812_06007_gb300 import binding as B
    from paper_1812_06007_gb300 import build as Bld
    from paper_1812_06007_gb300 import workloads as W
    Bld.build()
    B.lib()
    dev = torch.device("cuda", torch.cuda.current_device())
    n = a.n if a.n != 16384 else 2048
    m, q, reorth = (a.m if a.m != a.n else n), a.q, a.reorth
    amode = {"mixed": "fp32", "fp32": "fp32", "fp64": "fp64", "fp64emu": "fp64emu"}.get(a.mode)
    if amode is None:
        raise SystemExit("--workload adjoint runs --mode fp32, fp64 or fp64emu")
    f32 = amode == "fp32"
    mode = {"fp32": B.PURL_MODE_FP32, "fp64": B.PURL_MODE_FP64, "fp64emu": B.PURL_MODE_FP64_EMU}[amode]
    dt = torch.float32 if f32 else torch.float64
    esz = 4 if f32 else 8
    A = W.gaussian_matrix_torch(m, n, 2048, device=dev).to(dt).t().contiguous().t()
    gen = torch.Generator(device=dev)
    gen.manual_seed(W.SEED_B)
    Ub = torch.randn(n, m, generator=gen, device=dev, dtype=torch.float64).to(dt).t()
    Rb = torch.randn(n, n, generator=gen, device=dev, dtype=torch.float64).to(dt).t()
    Vb = torch.randn(n, n, generator=gen, device=dev, dtype=torch.float64).to(dt).t()
    nbytes = (B.purl_urv_backward_f32_workspace_bytes(m, n, q, mode) if f32 else
              B.purl_urv_backward_ex_workspace_bytes(m, n, q, mode))
    ws = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    Ab = B.empty_colmajor(m, n, dev, dt)
    stream = torch.cuda.current_stream()
    backward = B.purl_urv_backward_f32 if f32 else B.purl_urv_backward_ex

    def step():
        backward(A, q, reorth, W.SEED_G, Ub, Rb, Vb, mode=mode, out=Ab, workspace=ws, stream=stream)

    for _ in range(a.warmup):
        step()
    torch.cuda.synchronize()
    B.purl_profile_reset()
    B.purl_profile_set_stride(8)
    B.purl_profile_enable(True)
    launches0 = B.purl_launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(dev.index) as clk:
        e0.record(stream)
        for _ in range(a.steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
    launches = B.purl_launch_count() - launches0
    named = B.purl_profile_read_named()
    B.purl_profile_enable(False)
    sec = e0.elapsed_time(e1) / a.steps * 1e-3
    F = adjoint_flops(m, n, q, reorth)
    clocks = clk.summary()
    roof = roofline(None, named, a.steps, amode, sm_mhz=clocks.get("sm_mhz"),
                    sms=torch.cuda.get_device_properties(dev).multi_processor_count)
    # end to end: A and cotangents from pinned host memory, gradient back
    hA, hU = A.cpu().pin_memory(), Ub.cpu().pin_memory()
    hR, hV, hAb = Rb.cpu().pin_memory(), Vb.cpu().pin_memory(), torch.empty_like(Ab.cpu()).pin_memory()
    dA, dU, dR, dV = (B.empty_colmajor(*t.shape, dev, dt) for t in (A, Ub, Rb, Vb))
    x0, x1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    x0.record(stream)
    for _ in range(max(1, min(a.steps, 3))):
        for d_, h_ in ((dA, hA), (dU, hU), (dR, hR), (dV, hV)):
            d_.copy_(h_, non_blocking=True)
        backward(dA, q, reorth, W.SEED_G, dU, dR, dV, mode=mode, out=Ab, workspace=ws, stream=stream)
        hAb.copy_(Ab, non_blocking=True)
    x1.record(stream)
    torch.cuda.synchronize()
    e2e_sec = x0.elapsed_time(x1) / max(1, min(a.steps, 3)) * 1e-3
    cpu = None
    if not a.no_cpu_baseline:
        cpu = _adjoint_cpu(n, q, reorth)
    line = {
        "metric": ADJOINT_METRIC, "value": sec, "unit": "s", "n_gpus": 1, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": sec * 1e3, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "data": "synthetic",
        "dtype": {"fp32": "f32 (4 bf16 slices, exact sums)", "fp64": "f64",
                  "fp64emu": "f64 (emulated: 8 bf16 slices, exact sums)"}[amode],
        "config": {"workload": f"PowerURV reverse mode m={m} n={n} q={q} reorth={int(reorth)} {amode}, "
                               "Gaussian A, random cotangents", "m": m, "n": n, "q": q, "reorth": reorth,
                   "mode": amode,
                   "l2": f"working set {8 * (6 * m * n + 12 * n * n) / 2**20:.0f} MiB > L2"},
        "tflops": F / sec / 1e12, "flops_per_step": F, "roofline": roof, "cpu_baseline": cpu,
        "e2e": {"value": e2e_sec, "unit": "s", "h2d_bytes_per_step": esz * (2 * m * n + 2 * n * n),
                "d2h_bytes_per_step": esz * m * n},
        "gpu_launches": int(launches), "clocks": clocks,
        "kernels_by_name": {k: {"launches": v["launches"], "ms_per_step": v["ms"] / a.steps}
                            for k, v in sorted(named.items(), key=lambda kv: -kv[1]["ms"])[:8]},
    }
    print(json.dumps(line), flush=True)
    return 0


def _adjoint_cpu(n_full, q, reorth, n_sample: int = 384):
    """The oracle's reverse mode on an n_sample square Gaussian matrix, scaled to n_full by n^3."""
    import numpy as np
    from oracle import adjoint as oadj
    from paper_1812_06007_gb300 import workloads as W
    A = W.gaussian_matrix_np(n_sample, n_sample, 2048)
    rng = np.random.default_rng(W.SEED_B)
    Ub, Rb, Vb = (rng.standard_normal((n_sample, n_sample)) for _ in range(3))
    t0 = time.perf_counter()
    oadj.urv_backward(A, q, reorth, W.SEED_G, Ub, Rb, Vb)
    t = time.perf_counter() - t0
    scale = (n_full / n_sample) ** 3
    return {"value": t * scale, "unit": "s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"oracle reverse mode at m=n={n_sample} ({t:.2f} s; C QR + numpy products), "
                      f"scaled by (n/{n_sample})^3 to n={n_full}"}


def run_adjoint_reference(a):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    n = a.n if a.n != 16384 else 2048
    vals = []
    cpu = None
    for _ in range(a.warmup + a.steps):
        cpu = _adjoint_cpu(n, a.q, a.reorth)
        vals.append(cpu["value"])
    value = statistics.median(vals[a.warmup:])
    cpu["value"] = value
    line = {"impl": "reference", "metric": ADJOINT_METRIC, "value": value, "unit": "s", "n_gpus": a.gpus,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": value * 1e3, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"PowerURV reverse mode m=n={n} q={a.q}", "l2": "n/a (CPU)"},
            "cpu_baseline": cpu, "e2e": {"value": value, "unit": "s", "h2d_bytes_per_step": 0,
                                         "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- rsvd -----
RSVD_METRIC = "randomized SVD (Section 6) seconds and TFLOP/s, FP64, m=n=8192, l=256, q=2 reorth"


def rsvd_flops(m, n, l, q, reorth):
    """Products 2 m n l per application of A or A^T ((2q + 2) of them), the
    Householder QRs with explicit Q (2 (2 r l^2 - 2 l^3 / 3) each: q of m x l and
    q of n x l when re-orthonormalised, one of m x l and one of n x l always),
    and the two final l x l products; the Jacobi sweeps are not counted."""
    qr = lambda r: 2.0 * (2.0 * r * l * l - 2.0 * l ** 3 / 3.0)
    f = (2 * q + 2) * 2.0 * m * n * l + qr(m) + qr(n) + 2.0 * (m + n) * l * l
    if reorth:
        f += q * (qr(m) + qr(n))
    return f


def run_rsvd(a):
    import torch
    from paper_1812_06007_gb300 import binding as B
    from paper_1812_06007_gb300 import build as Bld
    from paper_1812_06007_gb300 import workloads as W
    Bld.build()
    B.lib()
    dev = torch.device("cuda", torch.cuda.current_device())
    n = a.n if a.n != 16384 else 8192
    m = a.m if a.m != a.n else n
    l, q, reorth = a.rank, a.q, a.reorth
    A = W.test_matrix_torch(m, n, W.sigma_profile("exponential", n, decades=6), device=dev)
    ws = torch.empty(B.purl_rsvd_workspace_bytes(m, n, l), dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    for _ in range(a.warmup):
        U, S, V = B.purl_rsvd(A, l, q, W.SEED_G, reorth, workspace=ws, stream=stream)
    torch.cuda.synchronize()
    B.purl_profile_reset()
    B.purl_profile_set_stride(8)
    B.purl_profile_enable(True)
    launches0 = B.purl_launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(dev.index) as clk:
        e0.record(stream)
        for _ in range(a.steps):
            U, S, V = B.purl_rsvd(A, l, q, W.SEED_G, reorth, workspace=ws, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
    launches = B.purl_launch_count() - launches0
    named = B.purl_profile_read_named()
    B.purl_profile_enable(False)
    sec = e0.elapsed_time(e1) / a.steps * 1e-3
    F = rsvd_flops(m, n, l, q, reorth)
    clocks = clk.summary()
    roof = roofline(None, named, a.steps, "fp64", sm_mhz=clocks.get("sm_mhz"),
                    sms=torch.cuda.get_device_properties(dev).multi_processor_count)
    # accuracy against the exact spectrum of the synthetic matrix (sigma_j prescribed)
    sig = torch.as_tensor(W.sigma_profile("exponential", n, decades=6)[:l], device=dev)
    sv_err = float(((S - sig).abs() / sig[0]).max())
    hA = A.cpu().pin_memory()
    dA = B.empty_colmajor(m, n, dev)
    x0, x1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    x0.record(stream)
    dA.copy_(hA, non_blocking=True)
    U, S, V = B.purl_rsvd(dA, l, q, W.SEED_G, reorth, workspace=ws, stream=stream)
    hU, hS, hV = U.cpu(), S.cpu(), V.cpu()
    x1.record(stream)
    torch.cuda.synchronize()
    e2e_sec = x0.elapsed_time(x1) * 1e-3
    cpu = None
    if not a.no_cpu_baseline:
        cpu = _rsvd_cpu(m, n, l, q, reorth)
    line = {
        "metric": RSVD_METRIC, "value": sec, "unit": "s", "n_gpus": 1, "steps": a.steps, "warmup": a.warmup,
        "ms_per_step": sec * 1e3, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"randomized SVD m={m} n={n} l={l} q={q} reorth={int(reorth)}, "
                               "sigma 10^(-6(j-1)/(n-1)), Haar-like factors", "m": m, "n": n, "l": l, "q": q,
                   "reorth": reorth, "l2": f"inputs larger than L2 (A is {8 * m * n / 2**20:.0f} MiB)"},
        "tflops": F / sec / 1e12, "flops_per_step": F,
        "errors": {"max_abs_sigma_err_rel_sigma1": sv_err},
        "roofline": roof, "cpu_baseline": cpu,
        "e2e": {"value": e2e_sec, "unit": "s", "h2d_bytes_per_step": 8 * m * n,
                "d2h_bytes_per_step": 8 * (m * l + l + n * l)},
        "gpu_launches": int(launches), "clocks": clocks,
        "kernels_by_name": {k: {"launches": v["launches"], "ms_per_step": v["ms"] / a.steps}
                            for k, v in sorted(named.items(), key=lambda kv: -kv[1]["ms"])[:8]},
    }
    print(json.dumps(line), flush=True)
    return 0


def _rsvd_cpu(m_full, n_full, l_full, q, reorth, n_sample: int = 768):
    """The oracle's RSVD on a scaled-down problem (m = n = n_sample, l scaled), scaled by m n l."""
    from oracle import rsvd as orsvd
    from paper_1812_06007_gb300 import workloads as W
    ls = max(1, int(round(l_full * n_sample / n_full)))
    A = W.test_matrix_np(n_sample, n_sample, W.sigma_profile("exponential", n_sample, decades=6))
    t0 = time.perf_counter()
    orsvd.rsvd(A, ls, q, W.SEED_G, reorth)
    t = time.perf_counter() - t0
    scale = (m_full * n_full * l_full) / (n_sample * n_sample * ls)
    return {"value": t * scale, "unit": "s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"oracle RSVD at m=n={n_sample}, l={ls} ({t:.2f} s; C QR + numpy products and SVD), "
                      f"scaled by m n l to the full problem"}


def run_rsvd_reference(a):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    n = a.n if a.n != 16384 else 8192
    vals, cpu = [], None
    for _ in range(a.warmup + a.steps):
        cpu = _rsvd_cpu(n, n, a.rank, a.q, a.reorth)
        vals.append(cpu["value"])
    value = statistics.median(vals[a.warmup:])
    cpu["value"] = value
    line = {"impl": "reference", "metric": RSVD_METRIC, "value": value, "unit": "s", "n_gpus": a.gpus,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": value * 1e3, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"randomized SVD m=n={n} l={a.rank} q={a.q}", "l2": "n/a (CPU)"},
            "cpu_baseline": cpu, "e2e": {"value": value, "unit": "s", "h2d_bytes_per_step": 0,
                                         "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------- product -----
def run_product(a):
    """One product engine on its own (the a2/a3/a6 products of Section 3): C = A B with m = n = k = a.n,
    FP64 operands resident on the device, the engine chosen by --engine.  Used for per-engine rooflines
    and ncu captures; not a PowerURV metric."""
    import torch
    from paper_1812_06007_gb300 import binding as B
    from paper_1812_06007_gb300 import build as Bld
    Bld.build()
    B.lib()
    dev = torch.device("cuda", torch.cuda.current_device())
    n = a.n
    k = a.k if a.k > 0 else n
    g = torch.Generator(device=dev)
    g.manual_seed(5)
    A = torch.randn(k, n, generator=g, device=dev, dtype=torch.float64).t()
    Bm = torch.randn(n, k, generator=g, device=dev, dtype=torch.float64).t()
    C = B.empty_colmajor(n, n, dev)
    C.zero_()
    stream = torch.cuda.current_stream()
    S = a.slices
    # --update: C <- C - A B (the trailing-update form: FP64 read-modify-write of C)
    alpha, beta = (-1.0, 1.0) if a.update else (1.0, 0.0)

    def step():
        if a.engine == "f64":
            B.purl_gemm_f64("N", "N", A, Bm, alpha=alpha, beta=beta, C=C, stream=stream)
        else:
            B.purl_gemm_tc("N", "N", A, Bm, alpha=alpha, beta=beta, C=C, slices=S, exact=(a.engine == "tcx"),
                           stream=stream)

    for _ in range(a.warmup):
        step()
    torch.cuda.synchronize()
    B.purl_profile_reset()
    B.purl_profile_set_stride(1)
    B.purl_profile_enable(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(dev.index) as clk:
        e0.record(stream)
        for _ in range(a.steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
    named = B.purl_profile_read_named()
    B.purl_profile_enable(False)
    ms = e0.elapsed_time(e1) / a.steps
    clocks = clk.summary()
    roof = roofline(None, named, a.steps, a.engine, sm_mhz=clocks.get("sm_mhz"),
                    sms=torch.cuda.get_device_properties(dev).multi_processor_count)
    if roof is not None:
        attach_traffic(roof)
    err = None
    if n <= 8192 and not a.update:
        ref = A @ Bm
        err = float((C - ref).abs().max() / (A.abs() @ Bm.abs()).max())
    form = "C = C - A B" if a.update else "C = A B"
    line = {"metric": f"product {form} ({a.engine}, slices={S if a.engine != 'f64' else 0})",
            "value": 2.0 * n * n * k / (ms * 1e-3) / 1e12,
            "unit": "TFLOP/s", "n_gpus": 1, "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "data": "synthetic",
            "dtype": "f64" if a.engine == "f64" else "bf16 slices",
            "config": {"workload": f"product m=n={n} k={k} {form} engine={a.engine} slices={S}",
                       "l2": f"operands larger than L2 ({8 * n * n / 2**20:.0f} MiB each)" if 8 * n * n > 129e6
                       else "operands fit in L2"},
            "max_rel_err": err, "clocks": clocks, "roofline": roof,
            "kernels_ms_per_step": {k: v["ms"] / a.steps for k, v in named.items()}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    a = parse()
    if a.workload == "product":
        return run_product(a)
    if a.workload == "batched":
        return run_batched_reference(a) if a.impl == "reference" else run_batched(a)
    if a.workload == "adjoint":
        return run_adjoint_reference(a) if a.impl == "reference" else run_adjoint(a)
    if a.workload == "rsvd":
        return run_rsvd_reference(a) if a.impl == "reference" else run_rsvd(a)
    if a.impl == "reference":
        return run_reference(a)
    return run_ours(a)


if __name__ == "__main__":
    sys.exit(main())
