"""PowerURV as a differentiable torch operation (FP64, G fixed by the seed).

``urv(A, q, reorth, seed)`` returns (U, R, V) with A = U R V^T (Section 3,
Eqs. (5)-(6)); its backward calls the library's hand-written reverse mode
``purl_urv_backward``, which recomputes the power iterates from A and the
seed and runs the chain rule through every product and QR on the GPU.  The
paper defines no derivative; the reverse rule is the standard one for a thin
QR with a positive R diagonal, stated in ``include/purl.h``.

``truncated_loss(A, q, reorth, seed, k, B)`` is L = ||A_k - B||_F^2 with the
rank-k truncation A_k = U(:,1:k) R(1:k,:) V^T of Section 5; the truncation
and the squared norm are composed from torch operations on (U, R, V), so its
gradient flows into the same backward.
"""
from __future__ import annotations

import torch

from . import binding


class PowerURV(torch.autograd.Function):
    @staticmethod
    def forward(ctx, A, q: int, reorth: bool, seed: int):
        A = binding.as_colmajor(A)
        U, R, V = binding.purl_urv_factor(A, q, reorth, seed, binding.PURL_MODE_FP64)
        ctx.save_for_backward(A)
        ctx.q, ctx.reorth, ctx.seed = q, reorth, seed
        return U, R, V

    @staticmethod
    def backward(ctx, Ubar, Rbar, Vbar):
        (A,) = ctx.saved_tensors
        m, n = A.shape
        cot = []
        for g, rows in ((Ubar, m), (Rbar, n), (Vbar, n)):
            cot.append(binding.as_colmajor(g) if g is not None else
                       torch.zeros((n, rows), dtype=torch.float64, device=A.device).t())
        Abar = binding.purl_urv_backward(A, ctx.q, ctx.reorth, ctx.seed, *cot)
        return Abar, None, None, None


def urv(A, q: int, reorth: bool, seed: int):
    """(U, R, V) of PowerURV in FP64; differentiable with respect to A."""
    return PowerURV.apply(A, q, reorth, seed)


def truncated_loss(A, q: int, reorth: bool, seed: int, k: int, B):
    """||U(:,1:k) R(1:k,:) V^T - B||_F^2 on the PowerURV factors of A."""
    U, R, V = urv(A, q, reorth, seed)
    Ak = U[:, :k] @ R[:k, :] @ V.t()
    return ((Ak - B) ** 2).sum()
