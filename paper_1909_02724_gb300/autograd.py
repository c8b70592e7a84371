"""Differentiable operators over the C-ABI kernels.

* ``backproject(Q, plan)``: Algorithm 4 (the packed kernel where the plan
  has one, else ``ifdk_backproject``; the same operator up to FP32 rounding);
  its backward is ``ifdk_project`` (the exact transpose of the back-projection
  matrix).
* ``project(vol, plan)``: the adjoint projector; its backward is the
  back-projection above.
* ``filter(E, plan)``: Algorithm 1 in FP32; its backward is
  ``ifdk_filter_adjoint`` (F_cos . T with T symmetric, because h is even).

All three are linear, so their backward passes need no saved tensors; only
the plan is kept.  ``unrolled_gd`` runs gradient-descent reconstruction on
|| A x - y ||^2 with A = project, recomputing each step in the backward pass
(``torch.utils.checkpoint``) instead of storing one volume per step.
"""
from __future__ import annotations

import torch
from torch.utils.checkpoint import checkpoint

from .binding import Plan


def _f32(t: torch.Tensor) -> torch.Tensor:
    if t.dtype != torch.float32:
        raise TypeError("the differentiable operators take float32 tensors")
    return t.contiguous()


def _backproject(plan: Plan, Q: torch.Tensor) -> torch.Tensor:
    """Back-projection of all views: packed views (ifdk_pack_views +
    ifdk_backproject_packed) where the plan has them, else ifdk_backproject."""
    if plan.has_packed(torch.float32):
        return plan.backproject_packed(plan.pack(Q))
    return plan.backproject(Q)


class BackprojectFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, Q, plan: Plan):
        ctx.plan = plan
        return _backproject(plan, _f32(Q))

    @staticmethod
    def backward(ctx, g_vol):
        if not ctx.needs_input_grad[0]:
            return None, None
        return ctx.plan.project(_f32(g_vol)), None


class ProjectFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, vol, plan: Plan):
        ctx.plan = plan
        return plan.project(_f32(vol))

    @staticmethod
    def backward(ctx, g_P):
        if not ctx.needs_input_grad[0]:
            return None, None
        return _backproject(ctx.plan, _f32(g_P)), None


class FilterFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, E, plan: Plan):
        ctx.plan = plan
        return plan.filter(_f32(E))

    @staticmethod
    def backward(ctx, g_Q):
        if not ctx.needs_input_grad[0]:
            return None, None
        return ctx.plan.filter_adjoint(_f32(g_Q)), None


def backproject(Q: torch.Tensor, plan: Plan) -> torch.Tensor:
    return BackprojectFn.apply(Q, plan)


def project(vol: torch.Tensor, plan: Plan) -> torch.Tensor:
    return ProjectFn.apply(vol, plan)


def filter(E: torch.Tensor, plan: Plan) -> torch.Tensor:  # noqa: A001 - the paper's stage name
    return FilterFn.apply(E, plan)


def fdk(E: torch.Tensor, plan: Plan) -> torch.Tensor:
    """Differentiable FDK (FP32): backproject(filter(E))."""
    return backproject(filter(E, plan), plan)


def gd_step(x: torch.Tensor, y: torch.Tensor, alpha: torch.Tensor, plan: Plan) -> torch.Tensor:
    """x - alpha * A^T (A x - y) with A = project, A^T = backproject."""
    return x - alpha * backproject(project(x, plan) - y, plan)


def unrolled_gd(plan: Plan, y: torch.Tensor, x0: torch.Tensor, alphas: torch.Tensor,
                recompute: bool = True) -> torch.Tensor:
    """len(alphas) unrolled gradient-descent steps; with recompute=True each step
    is re-run during the backward pass instead of keeping its intermediates."""
    x = x0
    for t in range(alphas.shape[0]):
        if recompute and torch.is_grad_enabled():
            x = checkpoint(gd_step, x, y, alphas[t], plan, use_reentrant=False)
        else:
            x = gd_step(x, y, alphas[t], plan)
    return x
