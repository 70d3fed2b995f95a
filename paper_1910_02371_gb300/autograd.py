"""Differentiable objective of generalized CP completion for torch autograd.

``cp_completion_loss(pattern, factors, loss, lam)`` returns the objective of
eq. obj, f = sum_e phi(t_e, m_e) + lam sum_n ||A^(n)||_F^2, as a float64
scalar tensor that autograd can differentiate with respect to the factor
matrices.  Forward runs one pass of the fused gradient kernel in loss-only
mode (model entries computed on the fly, nothing stored).  Backward is written
by hand: it calls the same kernel for the gradients, Table 1 / Appendix A,
grad^(n) = MTTKRP(phi', n) + 2 lam A^(n), which recomputes each model entry
from the factor rows instead of reading saved ones, and scales by the
incoming gradient.
"""
from __future__ import annotations

import torch

from . import tc


class TcLossGrad(torch.autograd.Function):
    @staticmethod
    def forward(ctx, pattern_box, loss, lam, A0, A1, A2):
        p = pattern_box[0]
        A0, A1, A2 = (a.contiguous() for a in (A0, A1, A2))
        f, _ = tc.loss_grad(p, [A0, A1, A2], loss, lam, want_grad=False)
        ctx.save_for_backward(A0, A1, A2)
        ctx.pattern_box = pattern_box
        ctx.loss = loss
        ctx.lam = lam
        return f.reshape(())

    @staticmethod
    def backward(ctx, grad_out):
        A0, A1, A2 = ctx.saved_tensors
        p = ctx.pattern_box[0]
        _, g = tc.loss_grad(p, [A0, A1, A2], ctx.loss, ctx.lam, want_loss=False)
        # scale on the device (no host read of grad_out, so graph capture works)
        s = grad_out.reshape(()).to(g[0].dtype)
        for gi in g:
            gi.mul_(s)
        return None, None, None, g[0], g[1], g[2]


def cp_completion_loss(pattern: "tc.Pattern", factors, loss: str = "ls", lam: float = 0.0):
    """Objective of eq. obj at `factors` (three I_n x R tensors), differentiable."""
    if len(factors) != 3:
        raise ValueError("order-3 tensors only")
    return TcLossGrad.apply([pattern], loss, float(lam), *factors)
