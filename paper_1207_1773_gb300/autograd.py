"""torch.autograd.Function around the generalized eigensolver: the selected
eigenpairs (lambda_il..iu, X) of A x = lambda B x with X^H B X = I, and their
reverse-mode derivative with respect to the Hermitian A and B computed by the
library (gbhe_hegv_adjoint).  Plumbing only: the forward solve and every step
of the backward run in the CUDA library."""
from __future__ import annotations

import numpy as np
import torch

from . import gbhegv as G

_EPS = float(np.finfo(np.float64).eps)


def _colmajor_copy(t):
    """A column-major copy (never a view: the solver overwrites its inputs)."""
    out = torch.empty((t.shape[1], t.shape[0]), dtype=t.dtype, device=t.device).t()
    out.copy_(t.detach())
    return out


class GeneralizedEigh(torch.autograd.Function):
    """w, X = GeneralizedEigh.apply(A, B, il, iu, nb): eigenvalues il..iu
    (1-based, ascending) and B-orthonormal eigenvectors.  A and B are complex128
    CUDA tensors, read from their lower triangles.  When a gradient is needed
    the forward solves for the whole spectrum (the derivative sums over it)
    and returns the selected part.  The eigenvector phase is free: losses must
    not depend on it."""

    @staticmethod
    def forward(ctx, A, B, il, iu, nb=0):
        n = A.shape[0]
        need = ctx.needs_input_grad[0] or ctx.needs_input_grad[1]
        Ac, Bc = _colmajor_copy(A), _colmajor_copy(B)
        if need:
            w_all, X_all = G.hegv(Ac, Bc, 1, n, nb=nb)
            w, X = w_all[il - 1:iu], X_all[:, il - 1:iu]
            ctx.save_for_backward(w_all, X_all)
        else:
            w, X = G.hegv(Ac, Bc, il, iu, nb=nb)
        ctx.il, ctx.iu = il, iu
        return w.clone(), X.clone()

    @staticmethod
    def backward(ctx, gw, gX):
        w_all, X_all = ctx.saved_tensors
        n = X_all.shape[0]
        m = ctx.iu - ctx.il + 1
        if gw is None:
            gw = torch.zeros(m, dtype=torch.float64, device=X_all.device)
        if gX is None:
            gX = torch.zeros((m, n), dtype=torch.complex128, device=X_all.device).t()
        gX = _colmajor_copy(gX)
        # degenerate-gap masking: 1e3 n eps ||A'|| with ||A'|| = max |lambda|
        delta = 1e3 * n * _EPS * float(w_all.abs().max())
        dA, dB = G.hegv_adjoint(w_all, X_all, ctx.il, ctx.iu, gw.to(torch.float64), gX, delta)
        return dA, dB, None, None, None


def generalized_eigh(A, B, il=1, iu=None, nb=0):
    return GeneralizedEigh.apply(A, B, il, A.shape[0] if iu is None else iu, nb)
