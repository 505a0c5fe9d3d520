"""The per-source ELBO as a differentiable PyTorch function.

``SourceObjective(plan)(theta)`` returns L_s for every source of the plan at
``theta`` ([n, 27] float64 on the device; rows in plan order).  Backward runs
the library's gradient-only pass (the adjoint of the pixel term through the
rendered moments, recomputed on the patches: nothing per pixel is stored by
the forward pass).  Backward of that gradient, i.e. Hessian-vector products
and double backward, uses the library's dense per-source Hessian.  Neighbours
of the plan's sources stay at their current parameters.
"""
from __future__ import annotations

import torch

from . import celeste as cel


class SourceObjective:
    def __init__(self, plan: cel.Plan):
        self.plan = plan
        self.rows = torch.as_tensor(plan.sources, dtype=torch.long, device=plan.dprob.theta.device)

    def load(self, theta: torch.Tensor):
        if theta.shape != (self.plan.n, cel.N_THETA):
            raise ValueError(f"theta must be [{self.plan.n}, {cel.N_THETA}]")
        self.plan.dprob.theta.index_copy_(0, self.rows, theta.detach().to(torch.float64))

    def __call__(self, theta: torch.Tensor) -> torch.Tensor:
        return _Elbo.apply(theta, self)


class _Elbo(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta, obj):
        obj.load(theta)
        e, _ = cel.elbo(obj.plan)
        ctx.save_for_backward(theta)
        ctx.obj = obj
        return e

    @staticmethod
    def backward(ctx, g_out):
        (theta,) = ctx.saved_tensors
        g = _Grad.apply(theta, ctx.obj)
        return g_out[:, None] * g, None


class _Grad(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta, obj):
        obj.load(theta)
        _, _, g = cel.elbo_grad(obj.plan)
        ctx.save_for_backward(theta)
        ctx.obj = obj
        return g

    @staticmethod
    def backward(ctx, g_out):
        (theta,) = ctx.saved_tensors
        obj = ctx.obj
        obj.load(theta)
        _, _, _, H = cel.elbo_grad_hess(obj.plan)
        return torch.einsum("nij,nj->ni", H, g_out), None
