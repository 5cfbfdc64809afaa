"""Packed device storage for the batched FP32 engine (``purl_urv_factor_batched``).

``Batch`` holds many column-major FP32 matrices back to back in one device
buffer (each with leading dimension m), allocates the packed U, R, V outputs
and the device array of ``purl_batch_item`` descriptors.  Matrices are put in
the descriptor array costliest first (largest m n^2), which is the order the
persistent kernel takes them in; ``order[i]`` is the caller's index of
descriptor i.  Marshalling only: all arithmetic runs in the library.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import binding


def _offsets(sizes):
    # 64-float (256-byte) aligned offsets
    off, out = 0, []
    for s in sizes:
        out.append(off)
        off += (int(s) + 63) // 64 * 64
    return np.array(out, dtype=np.int64), off


class Batch:
    def __init__(self, ms, ns, seeds, device="cuda"):
        import torch
        self.ms = np.asarray(ms, dtype=np.int64)
        self.ns = np.asarray(ns, dtype=np.int64)
        self.seeds = np.asarray(seeds, dtype=np.uint64)
        self.count = len(self.ms)
        if np.any(self.ns < 1) or np.any(self.ms < self.ns):
            raise ValueError("every matrix needs 1 <= n <= m")
        self.max_m = int(self.ms.max()) if self.count else 1
        self.max_n = int(self.ns.max()) if self.count else 1
        self.order = np.argsort(-(self.ms * self.ns * self.ns), kind="stable")
        self.a_off, a_total = _offsets(self.ms * self.ns)
        self.r_off, r_total = _offsets(self.ns * self.ns)
        f32 = torch.float32
        self.A = torch.zeros(max(a_total, 1), dtype=f32, device=device)
        self.U = torch.zeros(max(a_total, 1), dtype=f32, device=device)
        self.R = torch.zeros(max(r_total, 1), dtype=f32, device=device)
        self.V = torch.zeros(max(r_total, 1), dtype=f32, device=device)
        items = (binding.BatchItem * max(self.count, 1))()
        for d, i in enumerate(self.order):
            m, n = int(self.ms[i]), int(self.ns[i])
            it = items[d]
            it.m, it.n, it.lda, it.ldu, it.ldr, it.ldv = m, n, m, m, n, n
            it.A = self.A.data_ptr() + 4 * int(self.a_off[i])
            it.U = self.U.data_ptr() + 4 * int(self.a_off[i])
            it.R = self.R.data_ptr() + 4 * int(self.r_off[i])
            it.V = self.V.data_ptr() + 4 * int(self.r_off[i])
            it.seed = int(self.seeds[i])
        raw = bytes(memoryview(items).cast("B"))
        self.items = torch.frombuffer(bytearray(raw), dtype=torch.uint8).to(device)
        self.workspace = None

    # -- host <-> device of single matrices (column-major views) --
    def _view(self, buf, off, rows, cols):
        return buf[off:off + rows * cols].view(cols, rows).t()

    def a(self, i):
        return self._view(self.A, int(self.a_off[i]), int(self.ms[i]), int(self.ns[i]))

    def u(self, i):
        return self._view(self.U, int(self.a_off[i]), int(self.ms[i]), int(self.ns[i]))

    def r(self, i):
        return self._view(self.R, int(self.r_off[i]), int(self.ns[i]), int(self.ns[i]))

    def v(self, i):
        return self._view(self.V, int(self.r_off[i]), int(self.ns[i]), int(self.ns[i]))

    def set_a(self, i, A_host):
        import torch
        self.a(i).copy_(torch.from_numpy(np.asarray(A_host, dtype=np.float32)))

    def load_packed_a(self, host_packed):
        """Copy a host float32 array laid out like self.A (see pack_host) in one transfer."""
        import torch
        self.A.copy_(torch.from_numpy(host_packed))

    def pack_host(self, mats):
        """Host float32 array with matrix i (caller order) at its packed offset."""
        out = np.zeros(self.A.numel(), dtype=np.float32)
        for i, X in enumerate(mats):
            m, n = int(self.ms[i]), int(self.ns[i])
            out[self.a_off[i]:self.a_off[i] + m * n] = np.asarray(X, dtype=np.float32).reshape(-1, order="F")
        return out

    def ensure_workspace(self, variant: int = -1):
        import torch
        need = binding.purl_urv_batched_workspace_bytes(self.max_m, self.max_n, variant)
        if need == 0:
            raise RuntimeError("batched engine cannot run these sizes")
        if self.workspace is None or self.workspace.numel() < need:
            self.workspace = torch.empty(need, dtype=torch.uint8, device=self.A.device)
        return self.workspace

    def factor(self, q: int, reorth: bool = True, variant: int = -1, stream=None):
        ws = self.ensure_workspace(-1)
        binding.purl_urv_factor_batched(self.items, self.count, self.max_m, self.max_n, q, reorth, ws,
                                        variant=variant, stream=stream)

    def autotune(self, q: int, reorth: bool = True, stream=None):
        ws = self.ensure_workspace(-1)
        return binding.purl_urv_batched_autotune(self.items, self.count, self.max_m, self.max_n, q, reorth, ws,
                                                 stream=stream)

    def status(self, stream=None) -> int:
        return binding.purl_urv_batched_status(self.workspace, stream=stream)

    def item_view(self, d: int):
        """Device tensor slice of descriptor d alone (for per-matrix launches)."""
        return self.items[64 * d:64 * (d + 1)]


def flops(ms, ns, q: int, reorth: bool = True) -> float:
    """Algorithmic flops of PowerURV over a batch (explicit Q counted):
    2(2q+1) m n^2 for the products plus 2(2 r n^2 - 2 n^3 / 3) per QR of an
    r x n matrix (factor and form Q): q QRs of m x n and q of n x n when
    re-orthonormalised (the last being Eq. (5)'s), else one n x n, plus Eq. (6)'s."""
    m = np.asarray(ms, dtype=np.float64)
    n = np.asarray(ns, dtype=np.float64)
    qr = lambda r: 2.0 * (2.0 * r * n * n - 2.0 * n ** 3 / 3.0)
    gem = 2.0 * (2 * q + 1) * m * n * n
    if reorth and q > 0:
        tot = gem + q * qr(m) + q * qr(n) + qr(m)
    else:
        tot = gem + qr(n) + qr(m)
    return float(tot.sum())
