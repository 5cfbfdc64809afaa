"""Batched FP32 PowerURV (purl_urv_factor_batched) against the FP64 oracle.

Every matrix of the batch is factored by the oracle (Section 3, Eqs. (5)-(6),
FP64) from the same FP32 input and the same Philox key; the GPU computes in
FP32.  Bars, from FP32 arithmetic (u = 2^-24 ~ 6e-8) in Householder QR, whose
backward error is a small multiple of sqrt(m n) u:
  ||A - U R V^T||_F / ||A||_F <= 1e-5,  ||I - U^T U||_F, ||I - V^T V||_F <= 5e-5
  (n <= 256: about 1.5 n u and 3 n u; measured values sit 10x below),
  R upper triangular with a nonnegative diagonal,
  on the leading columns j that are determined -- two oracle runs agree to
  1e-3 there when G is perturbed elementwise and A normwise at the 1e-6
  level -- and whose FP32 error, sqrt(n) u (R_11/R_jj)^p with p = 1 with
  re-orthonormalisation and p = 2q without, stays below 1e-4: |R_jj| agrees
  with the oracle to 2e-3 relative plus 16 sqrt(n) u ||A||_2 absolute (the
  FP32 backward error), U(:,j) and V(:,j) to 2e-3.
The Gaussian draw in FP32 matches the FP64 one to a few FP32 ulps plus the
effect of rounding the two uniforms of each Box-Muller pair to FP32.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1812_06007_gb300 import workloads as W

pytestmark = pytest.mark.gpu
U32 = 2.0 ** -24


@pytest.fixture(scope="module")
def B():
    from paper_1812_06007_gb300 import binding, build
    build.build()
    return binding


def _batch(shapes, decades=6.0):
    from paper_1812_06007_gb300.batched import Batch
    ms = [s[0] for s in shapes]
    ns = [s[1] for s in shapes]
    b = Batch(ms, ns, [W.batched_seed(i) for i in range(len(shapes))])
    mats = [W.batched_matrix_np(m, n, i, decades) for i, (m, n) in enumerate(shapes)]
    b.load_packed_a(b.pack_host(mats))
    return b, mats


def _host(t):
    import torch
    torch.cuda.synchronize()
    return t.cpu().numpy().astype(np.float64)


def _determined_prefix(A, G, q, reorth, tol=1e-3, delta=1e-6):
    # FP32 rounding of the products acts like a normwise perturbation of the
    # iterates: model it by perturbing G elementwise and A normwise by delta.
    n = A.shape[1]
    rng = np.random.default_rng(99)
    Gp = G * (1.0 + delta * rng.standard_normal(G.shape))
    E = rng.standard_normal(A.shape)
    Ap = A + delta * np.linalg.norm(A) / np.linalg.norm(E) * E
    U0, R0, V0 = oracle.urv_g(A, G, q, reorth)
    U1, R1, V1 = oracle.urv_g(Ap, Gp, q, reorth)
    d0, d1 = np.abs(np.diag(R0)), np.abs(np.diag(R1))
    ok = (np.abs(d0 - d1) <= tol * d0) & (np.abs(V0 - V1).max(axis=0) <= tol) \
        & (np.abs(U0 - U1).max(axis=0) <= tol)
    J = int(np.argmin(ok)) if not ok.all() else n
    return J, (U0, R0, V0)


def _check_matrix(A, U, R, V, q, reorth, seed, with_oracle=True):
    m, n = A.shape
    assert np.linalg.norm(A - U @ R @ V.T) <= 1e-5 * np.linalg.norm(A)
    assert np.linalg.norm(np.eye(n) - U.T @ U) <= 5e-5
    assert np.linalg.norm(np.eye(n) - V.T @ V) <= 5e-5
    assert np.all(np.tril(R, -1) == 0.0)
    assert np.all(np.diag(R) >= 0.0)
    if not with_oracle:
        return
    J, (Uo, Ro, Vo) = _determined_prefix(A, oracle.gaussian(seed, n, n), q, reorth)
    # FP32 rounding reaches column j amplified by (R_11 / R_jj)^p: p = 1 when
    # every product and QR works on orthonormal iterates (each step loses
    # u ||A|| against sigma_j), p = 2q for the plain power iteration (Y_q is
    # rounded against sigma_1^2q while its j-th direction carries sigma_j^2q).
    # Compare columns whose amplified error sqrt(n) u (R_11/R_jj)^p <= 1e-4.
    p = 1 if (reorth or q == 0) else 2 * q
    do_all = np.diag(Ro)
    amp = np.sqrt(n) * U32 * (do_all[0] / np.maximum(do_all, 1e-300)) ** p
    K = min(J, int(np.argmin(amp <= 1e-4)) if not np.all(amp <= 1e-4) else n)
    d, do = np.diag(R)[:K], do_all[:K]
    # relative agreement plus the absolute backward-error term of FP32 QR
    # (a few sqrt(n) u ||A||_2; ||A||_2 = R_11 up to rounding)
    tol = 2e-3 * do + 16 * np.sqrt(n) * U32 * do_all[0]
    assert np.all(np.abs(d - do) <= tol), (K, np.max(np.abs(d - do) / tol))
    assert np.abs(U[:, :K] - Uo[:, :K]).max(initial=0.0) <= 2e-3
    assert np.abs(V[:, :K] - Vo[:, :K]).max(initial=0.0) <= 2e-3
    return K


def test_gaussian_f32_matches_oracle(B):
    # Box-Muller pairs (elements 2p, 2p+1 in column-major order) share
    # r = sqrt(-2 ln u0) and the angle 2 pi u1.  Rounding u0 to FP32 (relative
    # 2^-24) moves r by at most 2^-24 / r; rounding u1 moves the angle by at
    # most 2 pi 2^-24, i.e. r cos / r sin by 2 pi 2^-24 r.  On top of those,
    # a few FP32 ulps from logf, sincospif and the products.
    for rows, cols, seed in [(1, 1, 0), (7, 3, 5), (256, 256, W.batched_seed(3)), (33, 1000, 12345)]:
        G = _host(B.purl_gaussian_f32(seed, rows, cols)).reshape(-1, order="F")
        Go = oracle.gaussian(seed, rows, cols).reshape(-1, order="F")
        pad = np.concatenate([Go, np.zeros(len(Go) % 2)])
        r = np.repeat(np.hypot(pad[0::2], pad[1::2]), 2)[:len(Go)]
        bound = 8 * U32 * np.maximum(1.0, np.abs(Go)) + U32 / np.maximum(r, 1e-30) + 2 * np.pi * U32 * r
        assert np.all(np.abs(G - Go) <= bound)
        assert np.abs(G - Go).max() <= 1e-3


SHAPES = [(1, 1), (5, 1), (16, 16), (17, 17), (40, 33), (64, 64), (100, 70), (128, 100), (256, 130),
          (300, 256), (512, 256), (200, 200), (31, 16), (33, 32)]


@pytest.mark.parametrize("q,reorth", [(2, True), (0, True), (1, True), (1, False), (2, False), (3, True)])
def test_batched_matches_oracle(B, q, reorth):
    b, mats = _batch(SHAPES)
    b.factor(q, reorth)
    assert b.status() == 0
    Js = []
    for i, A in enumerate(mats):
        A = A.astype(np.float64)
        J = _check_matrix(A, _host(b.u(i)), _host(b.r(i)), _host(b.v(i)), q, reorth, W.batched_seed(i))
        Js.append(J)
    if reorth:  # with re-orthonormalisation the compared columns reach sigma_j ~ 2e-3
        assert min(K for K, (m, n) in zip(Js, SHAPES) if n >= 16) >= 6


def test_every_variant_and_autotune(B):
    b, mats = _batch(SHAPES[:10])
    outs = []
    for v in range(B.purl_urv_batched_variants()):
        if B.purl_urv_batched_workspace_bytes(b.max_m, b.max_n, v) == 0:
            continue
        b.factor(2, True, variant=v)
        assert b.status() == 0
        outs.append([_host(b.r(i)) for i in range(len(mats))])
        for i, A in enumerate(mats):
            _check_matrix(A.astype(np.float64), _host(b.u(i)), _host(b.r(i)), _host(b.v(i)), 2, True,
                          W.batched_seed(i), with_oracle=False)
    assert len(outs) >= 2
    # variants differ only in rounding order: leading diagonals agree to FP32 accuracy
    for o in outs[1:]:
        for i in range(len(mats)):
            d0, d1 = np.diag(outs[0][i]), np.diag(o[i])
            assert np.abs(d0[:4] - d1[:4]).max() <= 1e-4 * d0[0]
    v, ms = b.autotune(2, True)
    assert 0 <= v < B.purl_urv_batched_variants() and ms > 0
    b.factor(2, True)  # variant -1 takes the tuned one
    assert b.status() == 0


def test_per_matrix_launches_and_graph_replay_are_bitwise_equal(B):
    import torch
    b, mats = _batch(SHAPES[:8])
    b.factor(2, True, variant=1)
    ref = [(_host(b.u(i)), _host(b.r(i)), _host(b.v(i))) for i in range(len(mats))]
    # one launch per matrix (same device code, count = 1)
    b.U.zero_(); b.R.zero_(); b.V.zero_()
    ws = b.ensure_workspace(-1)
    for d in range(b.count):
        B.purl_urv_factor_batched(b.item_view(d), 1, b.max_m, b.max_n, 2, True, ws, variant=1)
    for i in range(len(mats)):
        for x, y in zip(ref[i], (_host(b.u(i)), _host(b.r(i)), _host(b.v(i)))):
            assert np.array_equal(x, y)
    # the same batched call captured in a CUDA graph and replayed
    b.U.zero_(); b.R.zero_(); b.V.zero_()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        b.factor(2, True, variant=1, stream=s)  # uncaptured first call on this stream
        torch.cuda.synchronize()
        b.U.zero_(); b.R.zero_(); b.V.zero_()
        torch.cuda.synchronize()
        with torch.cuda.graph(g, stream=s):
            b.factor(2, True, variant=1, stream=s)
    g.replay()
    torch.cuda.synchronize()
    for i in range(len(mats)):
        for x, y in zip(ref[i], (_host(b.u(i)), _host(b.r(i)), _host(b.v(i)))):
            assert np.array_equal(x, y)


def test_invalid_descriptor_is_skipped_and_reported(B):
    import torch
    from paper_1812_06007_gb300.binding import BatchItem
    b, mats = _batch(SHAPES[:4])
    raw = bytearray(b.items.cpu().numpy().tobytes())
    items = (BatchItem * b.count).from_buffer(raw)
    bad = int(np.where(b.order == 1)[0][0])  # descriptor of matrix 1
    items[bad].n = items[bad].m + 1           # n > m
    b.items.copy_(torch.frombuffer(raw, dtype=torch.uint8))
    b.factor(1, True)
    assert b.status() == B.PURL_ERR_UNSUPPORTED
    for i in (0, 2, 3):
        _check_matrix(mats[i].astype(np.float64), _host(b.u(i)), _host(b.r(i)), _host(b.v(i)), 1, True,
                      W.batched_seed(i), with_oracle=False)


def test_batched_argument_errors(B):
    L = B.lib()
    nul = ctypes.c_void_p(0)
    assert L.purl_urv_factor_batched(-1, nul, 8, 8, 1, 1, -1, nul, 0, nul) == -1
    assert L.purl_urv_factor_batched(2, nul, 8, 8, 1, 1, -1, nul, 0, nul) == -2
    assert L.purl_urv_factor_batched(0, nul, 2048, 8, 1, 1, -1, nul, 0, nul) == -3
    assert L.purl_urv_factor_batched(0, nul, 8, 16, 1, 1, -1, nul, 0, nul) == -4
    assert L.purl_urv_batched_workspace_bytes(4096, 16, -1) == 0
    assert L.purl_urv_factor_batched(0, nul, 8, 8, 1, 1, 99, nul, 0, nul) == -7


def test_config_4096_matrices(B):
    # 4096 matrices, n ~ U[16, 256], m ~ U[n, 2n], sigma_j = 10^(-6 (j-1)/(n-1)),
    # q = 2 with re-orthonormalisation, FP32: invariants on every matrix, the
    # oracle on a sample that includes the largest.
    import torch
    from paper_1812_06007_gb300.batched import Batch
    count = 4096
    ms, ns = W.batched_shapes(count)
    b = Batch(ms, ns, [W.batched_seed(i) for i in range(count)])
    mats = [W.batched_matrix_np(int(ms[i]), int(ns[i]), i) for i in range(count)]
    b.load_packed_a(b.pack_host(mats))
    b.autotune(2, True)
    b.factor(2, True)
    assert b.status() == 0
    # invariants on the device in FP64 (test-side products)
    worst_rec = worst_orth = 0.0
    for i in range(count):
        A = b.a(i).double()
        U, R, V = b.u(i).double(), b.r(i).double(), b.v(i).double()
        n = U.shape[1]
        worst_rec = max(worst_rec, float(torch.linalg.matrix_norm(A - U @ R @ V.t()) / torch.linalg.matrix_norm(A)))
        eye = torch.eye(n, dtype=torch.float64, device=A.device)
        worst_orth = max(worst_orth, float(torch.linalg.matrix_norm(eye - U.t() @ U)),
                         float(torch.linalg.matrix_norm(eye - V.t() @ V)))
        assert float(torch.tril(R, -1).abs().max()) == 0.0 if n > 1 else True
        assert float(torch.diagonal(R).min()) >= 0.0
    assert worst_rec <= 1e-5 and worst_orth <= 5e-5, (worst_rec, worst_orth)
    big = int(np.argmax(ms * ns * ns))
    for i in sorted({big, 0, 1, 2, 1000, 4095}):
        _check_matrix(mats[i].astype(np.float64), _host(b.u(i)), _host(b.r(i)), _host(b.v(i)), 2, True,
                      W.batched_seed(i))
