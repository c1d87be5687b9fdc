"""The subset objective f_s(x) = D_s(x) + (beta/n) S(x) of eq. 5 as a
torch.autograd.Function whose backward is the backprojection kernel plus the RDP
gradient kernel, scaled by the incoming gradient.

Modes (all run in the library's kernels; none keeps a sinogram-sized tensor unless
"store" is asked for):
  fused     forward computes f_s and its gradient in one pass over the subset's LORs
            and saves the image-sized gradient;
  recompute forward computes f_s only (projection + KL); backward projects again and
            backprojects (no sinogram-sized storage: for TOF data that would not fit
            beside a SAGA table);
  store     forward keeps A_s x (one subset sinogram); backward forms the KL ratio from
            it and backprojects without projecting again.
  auto      recompute when the subset sinogram exceeds `store_limit_bytes`, else fused.
"""
from __future__ import annotations

import numpy as np
import torch

from . import binding as pet


class SubsetObjective(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, plan, subset, prior, mode):
        ctx.plan, ctx.subset, ctx.prior, ctx.mode = plan, subset, prior, mode
        xd = x.detach().contiguous()
        if mode == "fused":
            obj, g = plan.objective_grad(xd, subset, prior=prior)
            ctx.save_for_backward(g)
        elif mode == "recompute":
            obj, _ = plan.objective_grad(xd, subset, prior=prior, obj_only=True)
            ctx.save_for_backward(xd)
        elif mode == "store":
            ax = plan.forward(xd, subset)
            obj, _ = plan.ratio(ax, subset, want_q=False)
            if prior is not None:  # the library adds (beta/n) S(x) onto the KL value
                pet.rdp(xd, plan.spacing, prior[1], prior[2], prior[0], prior[3] if len(prior) > 3 else None,
                        want_grad=False, want_hdiag=False, val_out=obj, accumulate_val=True)
            ctx.save_for_backward(xd, ax)
        else:
            raise ValueError(mode)
        return obj

    @staticmethod
    def backward(ctx, grad_out):
        plan, subset, prior, mode = ctx.plan, ctx.subset, ctx.prior, ctx.mode
        if mode == "fused":
            (g,) = ctx.saved_tensors
        elif mode == "recompute":
            (xd,) = ctx.saved_tensors
            _, g = plan.objective_grad(xd, subset, prior=prior, want_obj=False)
        else:
            xd, ax = ctx.saved_tensors
            _, q = plan.ratio(ax, subset, want_obj=False)
            g = plan.back(q, subset)
            if prior is not None:
                pet.rdp(xd, plan.spacing, prior[1], prior[2], prior[0], prior[3] if len(prior) > 3 else None,
                        want_hdiag=False, want_val=False, grad_out=g, accumulate=True)
        # chain rule with the scalar incoming gradient
        return g * grad_out.to(g.dtype), None, None, None, None


def subset_objective(x, plan, subset, beta=0.0, gamma=2.0, eps=1e-3, kappa=None, mode="auto",
                     store_limit_bytes=1 << 30):
    """f_s(x) (float64 0-d tensor) differentiable in x.  subset = -1: the full objective
    D(x) + beta S(x); otherwise D_s(x) + (beta/n) S(x)."""
    n = plan.nsub
    scale = beta if subset < 0 else beta / n
    prior = None if beta == 0 else ((scale, gamma, eps) if kappa is None else (scale, gamma, eps, kappa))
    if mode == "auto":
        shp = plan.subset_shape(subset) if subset >= 0 else plan.sino_shape
        mode = "recompute" if 4 * int(np.prod(shp)) > store_limit_bytes else "fused"
    return SubsetObjective.apply(x, plan, subset, prior, mode)
