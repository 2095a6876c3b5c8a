"""torch.autograd wrapper of the CL coefficient fit (forward / adjoint kernels).

Methods, "Coefficients learning on OMP": the learnable coefficients s are
masked by the support, passed through the fixed fully connected layer A to
give y' = A (s .* Mask), and learned by back-propagating the residual loss.
:class:`CLFit` exposes that layer with the loss L_b = 1/2 ||y_b - A_S s_S||^2
per signal: the forward runs ``clfit_forward`` (gather-GEMV over the support
columns of A), the backward runs ``clfit_adjoint`` (dL/ds_S = -A_S^T r).
Neither materialises A_S: both kernels index-gather the columns of A.
"""
from __future__ import annotations

import torch

from . import clfit_adjoint, clfit_forward


class CLFit(torch.autograd.Function):
    """loss = CLFit.apply(s, A, S, Y)

    s : (B, t) float32 coefficients on the support (differentiable)
    A : (m, n) float32 measurement matrix (column-major), fixed
    S : (B, t) int32 support indices, fixed
    Y : (m, B) float32 measurements, fixed
    returns the per-signal loss (B,).
    """

    @staticmethod
    def forward(ctx, s, A, S, Y):
        R, loss = clfit_forward(A, S, s.detach(), Y)
        ctx.save_for_backward(A, S, R)
        return loss

    @staticmethod
    def backward(ctx, gloss):
        A, S, R = ctx.saved_tensors
        g = clfit_adjoint(A, S, R)
        return g * gloss.to(g.dtype)[:, None], None, None, None
