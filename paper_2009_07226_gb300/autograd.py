"""Differentiable projector and TV-regularised reconstruction.

``Project`` and ``BackProject`` are ``torch.autograd.Function``s whose forward
and backward passes are the library's product kernels: the gradient of a
projection is a back projection with the stored transpose, and the reverse
(adjoint pair, Sec. III-B: the same kernel family serves both).  ``DataFit``
is the data term 0.5 ||A X - Y||^2 of Eq. 1 in library calls only (the
projection, then the residual with its squared norm, then in backward the
back projection of the residual).  ``TV`` wraps the fused smoothed-TV
kernel.  ``tv_reconstruct`` minimises 0.5 ||A X - Y||^2 + lam * TV_eps(X)
(Eq. 1 with R = lam * TV_eps) with Adam, every step on the GPU through these
Functions; ``xct_tv_reconstruct`` runs the same steps as one native loop.
"""
from __future__ import annotations

import torch

from . import xct


class Project(torch.autograd.Function):
    """y = A x (x [S, n, n] -> y [S, M, N_d]); backward: A^T grad."""

    @staticmethod
    def forward(ctx, x, plan):
        ctx.plan = plan
        return plan.project(x.contiguous())

    @staticmethod
    def backward(ctx, gy):
        return ctx.plan.backproject(gy.contiguous()), None


class BackProject(torch.autograd.Function):
    """x = A^T y (y [S, M, N_d] -> x [S, n, n]); backward: A grad."""

    @staticmethod
    def forward(ctx, y, plan):
        ctx.plan = plan
        return plan.backproject(y.contiguous())

    @staticmethod
    def backward(ctx, gx):
        return ctx.plan.project(gx.contiguous()), None


class DataFit(torch.autograd.Function):
    """sum over slices of 0.5 ||A x_s - y_s||^2 (FP64 scalar); backward:
    A^T (A x - y), scaled by the incoming gradient."""

    @staticmethod
    def forward(ctx, x, y, plan):
        q = plan.project(x.contiguous())
        r = torch.empty_like(q)
        val = torch.empty((), dtype=torch.float64, device=x.device)
        xct.xct_datafit(q, y.contiguous(), r, q[0].numel(), q.shape[0], val)
        ctx.plan = plan
        ctx.save_for_backward(r)
        return val

    @staticmethod
    def backward(ctx, g):
        (r,) = ctx.saved_tensors
        gx = ctx.plan.backproject(r)
        return (gx if _is_one(g) else gx * g.to(gx.dtype)), None, None


def _is_one(g) -> bool:
    return g is None or (g.numel() == 1 and float(g) == 1.0)


class TV(torch.autograd.Function):
    """sum over slices of weight * TV_eps(x_s), value and gradient in one
    fused kernel pass."""

    @staticmethod
    def forward(ctx, x, eps, weight):
        x = x.contiguous()
        S, n, _ = x.shape
        grad = torch.empty_like(x)
        val = torch.empty(S, dtype=torch.float64, device=x.device)
        xct.xct_tv(x, n, S, eps, weight, grad, val)
        ctx.save_for_backward(grad)
        return val.sum().to(x.dtype)

    @staticmethod
    def backward(ctx, g):
        (grad,) = ctx.saved_tensors
        return (grad if _is_one(g) else grad * g.to(grad.dtype)), None, None


def project(x, plan):
    return Project.apply(x, plan)


def backproject(y, plan):
    return BackProject.apply(y, plan)


def datafit(x, y, plan):
    return DataFit.apply(x, y, plan)


def tv(x, eps: float = 1e-3, weight: float = 1.0):
    return TV.apply(x, eps, weight)


def tv_reconstruct(plan, y, steps: int = 200, lr: float = 1e-2, lam: float = 1e-3,
                   eps: float = 1e-3, x0=None, history: bool = False):
    """Adam on 0.5 ||A x - y||^2 + lam TV_eps(x) from x0 (or 0); returns x
    (and the per-step loss values when history=True)."""
    x = (torch.zeros((y.shape[0], plan.n, plan.n), dtype=torch.float32, device=y.device)
         if x0 is None else x0.clone().float())
    m = torch.zeros_like(x)
    v = torch.zeros_like(x)
    losses = []
    for step in range(1, steps + 1):
        xr = x.detach().requires_grad_(True)
        loss = datafit(xr, y, plan) + tv(xr, eps, lam)
        (g,) = torch.autograd.grad(loss, xr)
        xct.xct_adam(x, g.contiguous(), m, v, x.numel(), lr, 0.9, 0.999, 1e-8, step)
        if history:
            losses.append(float(loss.detach()))
    return (x, losses) if history else x
