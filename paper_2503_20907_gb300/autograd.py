"""Differentiable projector: torch.autograd functions over a Plan.

The forward projection A and the adjoint A^T are linear and exact transposes
of each other (Sec. II.B: the backprojector is exactly matched), so the
gradient of the forward projection is the adjoint applied to the incoming
gradient, and the gradient of the adjoint is the forward projection.  Both
directions run the plan's CUDA kernels.
"""
from __future__ import annotations

import torch

from ._lib import Plan


class _Project(torch.autograd.Function):
    @staticmethod
    def forward(ctx, coef: torch.Tensor, plan: Plan) -> torch.Tensor:
        ctx.plan = plan
        return plan.fwd(coef.detach())

    @staticmethod
    def backward(ctx, grad_sino: torch.Tensor):
        return _Backproject.apply(grad_sino.contiguous(), ctx.plan), None


class _Backproject(torch.autograd.Function):
    @staticmethod
    def forward(ctx, sino: torch.Tensor, plan: Plan) -> torch.Tensor:
        ctx.plan = plan
        return plan.adj(sino.detach())

    @staticmethod
    def backward(ctx, grad_coef: torch.Tensor):
        return _Project.apply(grad_coef.contiguous(), ctx.plan), None


def project(coef: torch.Tensor, plan: Plan) -> torch.Tensor:
    """Forward projection p = A c of a [ny][nx] CUDA float32 coefficient image."""
    return _Project.apply(coef, plan)


def backproject(sino: torch.Tensor, plan: Plan) -> torch.Tensor:
    """Adjoint c' = A^T p of a CUDA float32 sinogram of plan.m values."""
    return _Backproject.apply(sino, plan)
