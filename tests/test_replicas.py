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
