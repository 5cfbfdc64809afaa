"""Multi-process path of bench.py on the CPU (gloo, world_size 2).

One matrix does not shard (replicas only): each rank factors its own matrix
and the benchmark combines ranks only through the max of their step times and
the whole-job rate N x flops / max time.  These tests run that host logic in
two gloo processes on 127.0.0.1; no GPU is involved.
"""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        local_ms = [120.0, 95.0][rank]
        mx = bench.max_over_ranks(local_ms)
        value = bench.replica_value(1e12, world, mx)
        q.put((rank, mx, value))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_weak_scaling_value():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, mx, value in out:
        assert mx == 120.0                         # the slowest rank sets the time
        assert value == pytest.approx(2 * 1e12 / 0.120 / 1e12)  # both ranks' work over it


def test_single_process_is_identity():
    import bench
    assert bench.max_over_ranks(7.5) == 7.5
    assert bench.replica_value(2e12, 1, 1000.0) == pytest.approx(2.0)


def test_flop_count_matches_table_1_reading():
    import bench
    n = 16384
    # q = 2, reorth: 10 n^3 (GEMMs) + 5 QRs of (8/3) n^3 = 23.33 n^3
    assert bench.urv_flops(n, n, 2, True) == pytest.approx((10 + 5 * 8 / 3) * n ** 3)
    # GEMM term 2(2q+1) m n^2 (Table 1 read with mn^2), no reorth: 2 QRs
    m = 3 * n
    assert bench.urv_flops(m, n, 1, False) == pytest.approx(6 * m * n * n + bench.qr_flops(n, n) + bench.qr_flops(m, n))


def test_roofline_picks_the_dominant_kernel_and_its_peak():
    import bench
    peaks, _ = bench._peaks()
    steps = 2
    named = {
        "tcx outer update": {"launches": 10, "ms": 500.0, "flops": 2.0e14, "bytes": 1e12},
        "panel_kernel": {"launches": 100, "ms": 300.0, "flops": 2.0e10, "bytes": 1e9},
        "split_exact_kernel": {"launches": 50, "ms": 100.0, "flops": 0.0, "bytes": 3e11},
    }
    r = bench.roofline(None, named, steps, "mixed")
    assert r["kernel"] == "tcx_gemm_kernel" and r["bound"] == "tensor"
    assert r["achieved"] == pytest.approx(2.0e14 / 0.5 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / peaks.get("bf16_tflops_sustained", 1700.0))
    assert r["launches_per_step"] == 5 and r["avg_launch_ms"] == pytest.approx(50.0)
    # FP64 kernels against the DFMA peak at the sampled clock (the panel of the FP64 modes), the
    # FP32 panel of the tensor-core modes against the FFMA peak, everything else against the copy
    # bandwidth
    named["tcx outer update"]["ms"] = 1.0
    r = bench.roofline(None, named, steps, "fp64emu", sm_mhz=1900.0, sms=152)
    assert r["kernel"] == "panel_kernel" and r["bound"] == "alu"
    assert r["peak"] == pytest.approx(152 * 4 * 1900e6 / 1e12)
    assert r["frac"] == pytest.approx(2.0e10 / 0.3 / 1e12 / r["peak"])
    r = bench.roofline(None, named, steps, "mixed", sm_mhz=1900.0, sms=152)
    assert r["kernel"] == "panel_kernel" and r["bound"] == "alu"
    assert r["peak"] == pytest.approx(152 * 128 * 2 * 1900e6 / 1e12)
    named["panel_kernel"]["ms"] = 1.0
    r = bench.roofline(None, named, steps, "mixed")
    assert r["kernel"] == "split_exact_kernel" and r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["achieved"] == pytest.approx(3e11 / 0.1 / 1e9)
    assert bench.roofline(None, {}, steps, "mixed") is None


def test_roofline_sums_call_sites_per_kernel_function():
    # no single call site of the exact engine beats the panel, but together they do
    import bench
    named = {
        "tcx outer update": {"launches": 10, "ms": 250.0, "flops": 1.0e14, "bytes": 1e12},
        "tcx outer C^T V~": {"launches": 10, "ms": 200.0, "flops": 0.8e14, "bytes": 1e12},
        "tcx inner update": {"launches": 100, "ms": 100.0, "flops": 0.1e14, "bytes": 1e11},
        "panel_kernel": {"launches": 100, "ms": 300.0, "flops": 2.0e10, "bytes": 1e9},
        "tc_gemm_kernel": {"launches": 4, "ms": 20.0, "flops": 2.0e13, "bytes": 1e10},
        "tc noalloc": {"launches": 1, "ms": 1.0, "flops": 1.0e12, "bytes": 1e9},
    }
    r = bench.roofline(None, named, 1, "mixed")
    assert r["kernel"] == "tcx_gemm_kernel"
    assert r["launches_per_step"] == 120
    assert r["achieved"] == pytest.approx(1.9e14 / 0.55 / 1e12)
    assert list(r["call_sites_ms_per_step"]) == ["tcx outer update", "tcx outer C^T V~", "tcx inner update"]
    funcs = bench.by_function(named)
    assert funcs["tc_gemm_kernel"]["launches"] == 5
    assert bench.kernel_function("tcx emu A Y") == "tcx_gemm_kernel"
    assert bench.kernel_function("split_exact_kernel") == "split_exact_kernel"
