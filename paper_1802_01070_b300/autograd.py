"""Differentiable projector and TV-regularised reconstruction with Adam.

``PctProject`` wraps the library's projector as a torch.autograd.Function:
forward computes y = A x with pct_forward, backward computes A^T g with
pct_adjoint; both recompute the proton paths (MLP and voxel walk) from the
loaded histories, so nothing about A is stored between them.  ``TotalVariation``
does the same for the isotropic TV of pct_tv.  ``reconstruct_tv_adam`` minimises
||A x - b||^2 + w TV(x) with the library's Adam kernel: a gradient-based
reconstruction beside the DROP solver of pct_solve.
"""
from __future__ import annotations

import torch


class PctProject(torch.autograd.Function):
    """y = A x for the protons loaded in ``ctx`` (a paper_1802_01070_b300.Context)."""

    @staticmethod
    def forward(fctx, x, ctx):
        fctx.pct = ctx
        return ctx.forward(x.detach().contiguous()).clone()

    @staticmethod
    def backward(fctx, g):
        return fctx.pct.adjoint(g.detach().contiguous()), None


class TotalVariation(torch.autograd.Function):
    """TV(x) = sum_v sqrt(|D+ x|_v^2 + eps^2) (float64 value) with its exact gradient."""

    @staticmethod
    def forward(fctx, x, ctx, eps):
        val, grad = ctx.tv(x.detach().contiguous(), eps)
        fctx.save_for_backward(grad)
        return val

    @staticmethod
    def backward(fctx, gout):
        (grad,) = fctx.saved_tensors
        return (gout.to(grad.dtype) * grad), None, None


def loss_and_grad(ctx, x, b, tv_weight=0.01, tv_eps=1e-6):
    """(loss float64, gradient) of ||A x - b||^2 + tv_weight TV(x) by autograd."""
    xv = x.detach().clone().requires_grad_(True)
    r = PctProject.apply(xv, ctx) - b
    loss = (r.double() ** 2).sum() + tv_weight * TotalVariation.apply(xv, ctx, tv_eps)
    loss.backward()
    return loss.detach(), xv.grad.detach()


def reconstruct_tv_adam(ctx, b, x0, steps=50, lr=1e-2, tv_weight=0.01, tv_eps=1e-6,
                        betas=(0.9, 0.999), adam_eps=1e-8, callback=None):
    """Minimise ||A x - b||^2 + tv_weight TV(x) from x0 with ``steps`` Adam steps.

    The Adam update runs in the library (pct_adam); returns (x, list of losses).
    """
    x = x0.detach().clone().contiguous()
    m = torch.zeros_like(x)
    v = torch.zeros_like(x)
    losses = []
    for t in range(1, steps + 1):
        loss, g = loss_and_grad(ctx, x, b, tv_weight, tv_eps)
        losses.append(loss)
        ctx.adam(x, g.contiguous(), m, v, t, lr=lr, beta1=betas[0], beta2=betas[1], eps=adam_eps)
        if callback is not None:
            callback(t, x, loss)
    return x, [float(l) for l in losses]
