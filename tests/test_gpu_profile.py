"""Per-kernel event timing (purl_profile_*): with a sampling stride the launch,
flop and byte counts still cover every launch and the scaled device time of a
kernel stays close to the fully timed one."""
import numpy as np
import pytest

from paper_1812_06007_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    from paper_1812_06007_gb300 import binding, build
    build.build()
    return binding


def _run(B, stride):
    import torch
    n = 1024
    A = W.test_matrix_torch(n, n, W.sigma_profile("exponential", n, decades=6), device="cuda")
    B.purl_urv_factor(A, 2, True, 7, mode=B.PURL_MODE_MIXED_BF16)
    torch.cuda.synchronize()
    B.purl_profile_reset()
    B.purl_profile_set_stride(stride)
    B.purl_profile_enable(True)
    l0 = B.purl_launch_count()
    for _ in range(2):
        B.purl_urv_factor(A, 2, True, 7, mode=B.PURL_MODE_MIXED_BF16)
    torch.cuda.synchronize()
    launches = B.purl_launch_count() - l0
    named = B.purl_profile_read_named()
    B.purl_profile_enable(False)
    B.purl_profile_set_stride(1)
    return launches, named


def test_sampled_timing_counts_every_launch(B):
    l1, full = _run(B, 1)
    l8, samp = _run(B, 8)
    assert l1 == l8 == sum(v["launches"] for v in full.values()) == sum(v["launches"] for v in samp.values())
    assert set(full) == set(samp)
    for k in full:
        assert full[k]["launches"] == samp[k]["launches"]
        assert full[k]["flops"] == samp[k]["flops"]
        assert samp[k]["ms"] > 0.0
    # the kernels that dominate the time are estimated to within a factor of 2
    top = sorted(full, key=lambda k: -full[k]["ms"])[:3]
    for k in top:
        assert 0.5 <= samp[k]["ms"] / full[k]["ms"] <= 2.0, (k, samp[k]["ms"], full[k]["ms"])
