"""PowerURV as a differentiable torch operation (G fixed by the seed).

``urv(A, q, reorth, seed)`` returns (U, R, V) with A = U R V^T (Section 3,
Eqs. (5)-(6)); its backward calls the library's hand-written reverse mode
``purl_urv_backward``, which recomputes the power iterates from A and the
seed and runs the chain rule through every product and QR on the GPU.  The
paper defines no derivative; the reverse rule is the standard one for a thin
QR with a positive R diagonal, stated in ``include/purl.h``.

``truncate(U, R, V, k)`` is the rank-k truncation A_k = U(:,1:k) R(1:k,:) V^T
of Section 5 computed by the library's ``purl_urv_truncate``; its backward
maps the cotangent of A_k to those of U, R, V with the library's FP64
product engine.  ``truncated_loss(A, q, reorth, seed, k, B)`` is
L = ||A_k - B||_F^2 on top of both.
"""
from __future__ import annotations

import torch

from . import binding


def _colmajor(x, dtype):
    """Column-major copy of x in `dtype` (no copy if already so)."""
    if x.dtype != dtype:
        x = x.to(dtype)
    if x.numel() == 0 or (x.stride(0) == 1 and x.stride(1) >= max(1, x.shape[0])):
        return x
    return x.t().contiguous().t()


class PowerURV(torch.autograd.Function):
    """Forward purl_urv_factor_ex (FP64 tensors) or purl_urv_factor_f32 (FP32
    tensors) in `mode`; backward the library's reverse mode in the same mode."""

    @staticmethod
    def forward(ctx, A, q: int, reorth: bool, seed: int, mode: int):
        f32 = A.dtype == torch.float32
        A = _colmajor(A, A.dtype if f32 else torch.float64)
        if f32:
            U, R, V = binding.purl_urv_factor_f32(A, q, reorth, seed, mode)
        else:
            U, R, V = binding.purl_urv_factor(A, q, reorth, seed, mode)
        ctx.save_for_backward(A)
        ctx.q, ctx.reorth, ctx.seed, ctx.mode, ctx.f32 = q, reorth, seed, mode, f32
        return U, R, V

    @staticmethod
    def backward(ctx, Ubar, Rbar, Vbar):
        (A,) = ctx.saved_tensors
        m, n = A.shape
        cot = []
        for g, rows in ((Ubar, m), (Rbar, n), (Vbar, n)):
            cot.append(_colmajor(g, A.dtype) if g is not None else
                       torch.zeros((n, rows), dtype=A.dtype, device=A.device).t())
        if ctx.f32:
            Abar = binding.purl_urv_backward_f32(A, ctx.q, ctx.reorth, ctx.seed, *cot, mode=ctx.mode)
        else:
            Abar = binding.purl_urv_backward_ex(A, ctx.q, ctx.reorth, ctx.seed, *cot, mode=ctx.mode)
        return Abar, None, None, None, None


def urv(A, q: int, reorth: bool, seed: int, mode: int | None = None):
    """(U, R, V) of PowerURV, differentiable with respect to A.  FP64 tensors
    default to PURL_MODE_FP64, FP32 tensors to PURL_MODE_FP32; the backward
    runs in the forward's mode (FP64, FP64_EMU or FP32)."""
    if mode is None:
        mode = binding.PURL_MODE_FP32 if A.dtype == torch.float32 else binding.PURL_MODE_FP64
    return PowerURV.apply(A, q, reorth, seed, mode)


class Truncate(torch.autograd.Function):
    """A_k = U(:,1:k) R(1:k,:) V^T; with Abar the cotangent of A_k:
    Ubar(:,1:k) = Abar V R(1:k,:)^T,  Rbar(1:k,:) = U(:,1:k)^T Abar V,
    Vbar = Abar^T U(:,1:k) R(1:k,:)  (zero elsewhere)."""

    @staticmethod
    def forward(ctx, U, R, V, k: int):
        ctx.dtype = U.dtype
        U, R, V = (binding.as_colmajor(x) for x in (U, R, V))  # FP64 (FP32 factors are widened)
        ctx.save_for_backward(U, R, V)
        ctx.k = k
        return binding.purl_urv_truncate(U, R, V, k).to(ctx.dtype)

    @staticmethod
    def backward(ctx, Abar):
        Ub, Rb, Vb = Truncate._cotangents(ctx, Abar)
        return Ub.to(ctx.dtype), Rb.to(ctx.dtype), Vb.to(ctx.dtype), None

    @staticmethod
    def _cotangents(ctx, Abar):
        U, R, V = ctx.saved_tensors
        k = ctx.k
        m, n = U.shape
        G = binding.as_colmajor(Abar)
        Ub = binding.empty_colmajor(m, n, U.device)
        Rb = binding.empty_colmajor(n, n, U.device)
        Ub.zero_()
        Rb.zero_()
        if k == 0:
            return Ub, Rb, torch.zeros_like(Rb)
        Uk, Rk = U[:, :k], R[:k, :]
        W = binding.purl_gemm_f64("N", "N", G, V)                      # Abar V       (m x n)
        binding.purl_gemm_f64("N", "T", W, Rk, C=Ub[:, :k])            # ... R_k^T    (m x k)
        binding.purl_gemm_f64("T", "N", Uk, W, C=Rb[:k, :])            # U_k^T Abar V (k x n)
        X = binding.purl_gemm_f64("N", "N", Uk, Rk)                    # U_k R_k      (m x n)
        Vb = binding.purl_gemm_f64("T", "N", G, X)                     # Abar^T X     (n x n)
        return Ub, Rb, Vb


def truncate(U, R, V, k: int):
    """Rank-k truncation U(:,1:k) R(1:k,:) V^T (Section 5) by the library; differentiable."""
    return Truncate.apply(U, R, V, k)


def truncated_loss(A, q: int, reorth: bool, seed: int, k: int, B, mode: int | None = None):
    """||U(:,1:k) R(1:k,:) V^T - B||_F^2 on the PowerURV factors of A (mode as for urv)."""
    U, R, V = urv(A, q, reorth, seed, mode)
    Ak = truncate(U, R, V, k)
    return ((Ak - B) ** 2).sum()
