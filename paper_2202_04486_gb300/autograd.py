"""Differentiable MDC: the forward operator as a torch.autograd.Function whose backward is the
hand-written adjoint kernel.

The MDC operator is linear (Eq. 1-3), so the vector-Jacobian product of U = P_B X is P_B^H applied to
the incoming gradient -- exactly the adjoint (the cross-correlation used by the gradient of Eq. 6).
Both directions run in the CUDA kernels behind the C ABI (mdc_forward / mdc_adjoint); this module only
wires them into autograd so that preconditioners (e.g. the reciprocity projection C_r of Eq. 4) and
regularisers written as torch operations compose with the operator.
"""
from __future__ import annotations

import torch

from .binding import MDCPlan


class MDCFunction(torch.autograd.Function):
    """U = MDC_B(X) for the sources idx; backward: grad_X = MDC_B^H(grad_U)."""

    @staticmethod
    def forward(ctx, X: torch.Tensor, plan: MDCPlan, idx: torch.Tensor) -> torch.Tensor:
        ctx.plan = plan
        ctx.save_for_backward(idx)
        return plan.forward(X.contiguous(), idx)

    @staticmethod
    def backward(ctx, grad_U: torch.Tensor):
        (idx,) = ctx.saved_tensors
        grad_X = ctx.plan.adjoint(grad_U.contiguous(), idx) if ctx.needs_input_grad[0] else None
        return grad_X, None, None


def mdc(X: torch.Tensor, plan: MDCPlan, idx: torch.Tensor) -> torch.Tensor:
    """Differentiable forward MDC of X ([nv][nr][nt], float32, CUDA) for the source batch idx."""
    return MDCFunction.apply(X, plan, idx)


def reciprocity(X: torch.Tensor) -> torch.Tensor:
    """Reciprocity preconditioner C_r of Eq. 4: 1/2 (X + X^T), T swapping receiver and virtual source."""
    return 0.5 * (X + X.transpose(0, 1))
