#!/usr/bin/env python
"""PowerURV throughput on one GB300 (or N replicas), printed as ONE JSON line.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--mode mixed|fp64] [--m M] [--n N] [--q Q] [--no-reorth]

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
    ap.add_argument("--mode", choices=["mixed", "fp64"], default="mixed")
    ap.add_argument("--m", type=int, default=0, help="rows (default n)")
    ap.add_argument("--n", type=int, default=16384)
    ap.add_argument("--q", type=int, default=2)
    ap.add_argument("--no-reorth", action="store_true")
    ap.add_argument("--cpu-sample-n", type=int, default=2560,
                    help="size of the oracle's bounded CPU sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-profile", action="store_true", help="skip per-kernel event timing")
    ap.add_argument("--fp64-n", type=int, default=8192,
                    help="size of the FP64-path comparison run (0 = skip); FP64 at n=16384 takes minutes")
    a = ap.parse_args()
    a.m = a.m or a.n
    a.reorth = not a.no_reorth
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
    mode = B.PURL_MODE_MIXED_BF16 if a.mode == "mixed" else B.PURL_MODE_FP64
    m, n, q, reorth = a.m, a.n, a.q, a.reorth

    sigma = W.sigma_profile("exponential", n, decades=6)
    A = W.test_matrix_torch(m, n, sigma, device=dev)
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
        B.purl_profile_reset()
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
    fp64 = None
    if a.mode == "mixed" and a.fp64_n > 0:
        del ws
        torch.cuda.empty_cache()
        fp64 = fp64_compare(a, dev, B, W, seed)

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return 0

    # ---- roofline of the dominant kernel class ----
    roof = roofline(prof, prof_named, a.steps, a.mode)
    if roof is not None and prof_named:
        roof["share_of_step"] = prof_named[roof["kernel"]]["ms"] / a.steps / ms_step
    cpu = None
    if not a.no_cpu_baseline and world == 1:
        v, t, cores = cpu_oracle_run(a.cpu_sample_n, q, reorth)
        cpu = {"value": v, "unit": "TFLOP/s", "cores": cores, "kind": "oracle",
               "sample": f"PowerURV m=n={a.cpu_sample_n} q={q} reorth={int(reorth)}, FP64 C oracle "
                         f"(OpenMP), one factorization, {t:.2f} s"}
    line = {
        "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16+f64" if a.mode == "mixed" else "f64", "data": "synthetic",
        "config": {"workload": f"PowerURV m={m} n={n} q={q} reorth={int(reorth)} {a.mode}",
                   "m": m, "n": n, "q": q, "reorth": reorth, "mode": a.mode,
                   "sigma": "10^(-6(j-1)/(n-1)), Haar factors", "parallelism": f"replicas{world}",
                   "l2": f"inputs larger than L2 (A is {8 * m * n / 2**30:.1f} GiB)"},
        "sec_per_factorization": ms_step * 1e-3,
        "fp64_path": fp64,
        "speedup_vs_fp64_path": (value / fp64["tflops"]) if fp64 else None,
        "flops_per_step": flops,
        "errors": errs,
        "roofline": roof,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": int(launches),
        "clocks": clk.summary(),
        "kernels": prof,
        "kernels_by_name": ({k: {"launches": v["launches"], "ms_per_step": v["ms"] / a.steps,
                                 "tflops": v["flops"] / max(v["ms"], 1e-9) / 1e9}
                             for k, v in sorted(prof_named.items(), key=lambda kv: -kv[1]["ms"])}
                            if prof_named else None),
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def fp64_compare(a, dev, B, W, seed):
    """Time the FP64 path (1 warm-up, 1 timed) at n = a.fp64_n on the same recipe."""
    import torch
    n = a.fp64_n
    m = n if a.m == a.n else int(round(a.m * n / a.n))
    A = W.test_matrix_torch(m, n, W.sigma_profile("exponential", n, decades=6), device=dev)
    U, R, V = B.empty_colmajor(m, n, dev), B.empty_colmajor(n, n, dev), B.empty_colmajor(n, n, dev)
    ws = torch.empty(B.purl_urv_workspace_bytes(m, n, B.PURL_MODE_FP64), dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    B.purl_urv_factor(A, a.q, a.reorth, seed, mode=B.PURL_MODE_FP64, out=(U, R, V), workspace=ws, stream=stream)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    B.purl_urv_factor(A, a.q, a.reorth, seed, mode=B.PURL_MODE_FP64, out=(U, R, V), workspace=ws, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    sec = e0.elapsed_time(e1) * 1e-3
    errs = probe_errors(A, U, R, V)
    return {"m": m, "n": n, "q": a.q, "reorth": a.reorth, "sec": sec,
            "tflops": urv_flops(m, n, a.q, a.reorth) / sec / 1e12, "errors": errs,
            "note": "FP64 path timed at this size (1 warm-up + 1 timed factorization); its TFLOP/s is the "
                    "FP64-pipe rate, which does not grow with n beyond this size"}


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
    import torch
    m, n = A.shape
    hA = torch.empty((n, m), dtype=torch.float64, pin_memory=True).t()
    hA.copy_(A)
    hU = torch.empty((n, m), dtype=torch.float64, pin_memory=True).t()
    hR = torch.empty((n, n), dtype=torch.float64, pin_memory=True).t()
    hV = torch.empty((n, n), dtype=torch.float64, pin_memory=True).t()
    dA = B.empty_colmajor(m, n, dev)
    stream = torch.cuda.current_stream()

    def step():
        dA.copy_(hA, non_blocking=True)
        B.purl_urv_factor(dA, a.q, a.reorth, seed, mode=mode, out=(U, R, V), workspace=ws, stream=stream)
        hU.copy_(U, non_blocking=True)
        hR.copy_(R, non_blocking=True)
        hV.copy_(V, non_blocking=True)

    step()
    torch.cuda.synchronize()
    steps = max(1, min(a.steps, 3))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = max_over_ranks(e0.elapsed_time(e1) / steps, dev)
    return {"value": urv_flops(m, n, a.q, a.reorth) * world / (ms * 1e-3) / 1e12, "unit": "TFLOP/s",
            "ms_per_step": ms, "h2d_bytes_per_step": 8 * m * n, "d2h_bytes_per_step": 8 * (m * n + 2 * n * n),
            "steps": steps}


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


# FP64 DFMA peak of this GPU, measured with a DFMA-loop kernel (2 DFMA/clk/SM
# x 152 SMs at the clock under load); MEASURED_PEAKS.json carries no FP64 figure.
FP64_DFMA_PEAK_TFLOPS = 1.20


def roofline(prof, named, steps, mode):
    """Roofline of the dominant kernel (by device time in the timed region).

    Tensor-core kernels: issued BF16 flops (2 m n k per slice pair) over their
    event-timed duration against the measured sustained BF16 peak; FP64 DFMA
    kernels: FP64 flops against the measured DFMA peak; everything else:
    algorithmic bytes against the measured copy bandwidth."""
    if not named:
        return None
    peaks, src = _peaks()
    name = max(named, key=lambda k: named[k]["ms"])
    st = named[name]
    if st["launches"] == 0 or st["ms"] <= 0:
        return None
    sec = st["ms"] * 1e-3
    base = {"kernel": name, "launches_per_step": st["launches"] / steps,
            "avg_launch_ms": st["ms"] / st["launches"], "traffic": None,
            "share_of_step": None, "hbm_gbs_algorithmic": st["bytes"] / sec / 1e9}
    if name.startswith("tc") or name == "tc_gemm_kernel":
        achieved = st["flops"] / sec / 1e12
        peak = peaks.get("bf16_tflops_sustained", 1700.0)
        base.update({"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "peak_source": f"{src} bf16 sustained (cuBLAS)",
                     "flops_counted": "issued: 2 m n k per BF16 slice pair"})
        return base
    if name in ("panel_kernel", "gemm_f64_kernel", "gram_kernel") or name.startswith("gemm_f64"):
        achieved = st["flops"] / sec / 1e12
        base.update({"bound": "alu", "achieved": achieved, "peak": FP64_DFMA_PEAK_TFLOPS, "unit": "TFLOP/s",
                     "frac": achieved / FP64_DFMA_PEAK_TFLOPS,
                     "peak_source": "measured FP64 DFMA loop, 2 DFMA/clk/SM x 152 SMs"})
        return base
    achieved = st["bytes"] / sec / 1e9
    peak = peaks.get("hbm_gbs", 6800.0)
    base.update({"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                 "peak_source": f"{src} hbm copy"})
    return base


def main():
    a = parse()
    if a.impl == "reference":
        return run_reference(a)
    return run_ours(a)


if __name__ == "__main__":
    sys.exit(main())
