"""Differentiable forward transform.

``nfft_bandlimited(fhat, x, plan)`` returns f = Psi F D_psihat fhat at the
nodes x (Eq. 4.11) and supports autograd with respect to both inputs:

* d f-hat:  grad_fhat = A^H grad_f, the adjoint transform (A = Psi F D_psihat
  is complex linear in fhat, so PyTorch's conjugate-Wirtinger convention
  gives the adjoint);
* d x:      grad_x[j, t] = sum_b Re(conj(grad_f[b, j]) * d f_{b,j} / d x_{j,t}),
  the node-derivative kernel (x is real, f complex).

All three products run in the library's kernels; this module only routes
tensors.  The plan's node state is re-set in backward if another call
changed it in between.
"""
from __future__ import annotations

import torch

from . import Plan

__all__ = ["NFFTBL", "nfft_bandlimited"]


class NFFTBL(torch.autograd.Function):
    @staticmethod
    def forward(ctx, fhat: torch.Tensor, x: torch.Tensor, plan: Plan):
        xs = x.detach().contiguous()
        plan.set_nodes(xs)
        token = object()
        plan._autograd_token = token
        f = plan.forward(fhat.detach().contiguous())
        ctx.save_for_backward(fhat.detach(), xs)
        ctx.plan = plan
        ctx.token = token
        return f

    @staticmethod
    def backward(ctx, grad_f: torch.Tensor):
        fhat, xs = ctx.saved_tensors
        plan: Plan = ctx.plan
        if getattr(plan, "_autograd_token", None) is not ctx.token:
            plan.set_nodes(xs)
            plan._autograd_token = ctx.token
        gf = grad_f.contiguous()
        grad_fhat = plan.adjoint(gf) if ctx.needs_input_grad[0] else None
        grad_x = plan.node_grad(fhat.contiguous(), gf) if ctx.needs_input_grad[1] else None
        return grad_fhat, grad_x, None


def nfft_bandlimited(fhat: torch.Tensor, x: torch.Tensor, plan: Plan) -> torch.Tensor:
    """Differentiable f = Psi F D_psihat fhat at nodes x (shape (B, N))."""
    return NFFTBL.apply(fhat, x, plan)
