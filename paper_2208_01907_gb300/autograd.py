"""Differentiable hybrid solve (adjoint through the same factorization).

``HybridSolve.apply(H, vals, b)`` factorizes K-bar (CSR values ``vals`` on the
pattern of ``H``), forms the Schur complement (Alg. 1) and returns x = K-bar^-1 b
(Alg. 2).  Backward: lam = K-bar^-T dJ/dx is one more hf_solve with the factor
kept by the context (K-bar is symmetric), dJ/db = lam, and dJ/dvals comes from
hf_values_adjoint (dJ/dK-bar_ij = -lam_i x_j).  Only the context (factor, X12,
S22 factors) and x are kept for the backward pass.

The context holds one factorization at a time.  The forward pass records the
context's factorization generation; a backward pass that finds the context
factorized again since then (another hybrid_solve on the same HybridFactor in
the same graph, or a deferred backward) raises instead of using the wrong factor.
Give each live graph node its own HybridFactor.
"""
from __future__ import annotations

import torch

from .hf import HybridFactor


class HybridSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, H: HybridFactor, vals: torch.Tensor, b: torch.Tensor, tau: float = 1e-2):
        if H.has_row_signs:
            # K-bar = J S is not symmetric: its transposed solve is J S^-1, not another hf_solve
            raise NotImplementedError("HybridSolve needs a symmetric K-bar (no row signs)")
        vals_c = vals.detach().contiguous()
        H.factorize(vals_c, tau)
        H.schur()
        bt = b.detach().reshape(-1, H.L).contiguous()          # (nrhs, L) = column-major L x nrhs
        x = torch.zeros_like(bt)
        H.solve(bt, x)
        ctx.H = H
        ctx.generation = H.generation
        ctx.b_shape = b.shape
        ctx.save_for_backward(x)
        return x.reshape(b.shape)

    @staticmethod
    def backward(ctx, gx):
        (x,) = ctx.saved_tensors
        H = ctx.H
        if H.generation != ctx.generation:
            raise RuntimeError("HybridSolve.backward: the HybridFactor was factorized again after this "
                               "forward pass (its factor no longer matches x); use one HybridFactor per "
                               "live hybrid_solve")
        g = gx.detach().reshape(-1, H.L).contiguous()
        lam = torch.zeros_like(g)
        H.solve(g, lam)                                      # K-bar^T = K-bar: the same factor
        gvals = torch.empty(H._col.shape[0], dtype=torch.float64, device=x.device)
        H.values_adjoint(x, lam, gvals)
        return None, gvals, lam.reshape(ctx.b_shape), None


def hybrid_solve(H: HybridFactor, vals: torch.Tensor, b: torch.Tensor, tau: float = 1e-2) -> torch.Tensor:
    return HybridSolve.apply(H, vals, b, tau)
