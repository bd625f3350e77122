"""torch.autograd.Function around the hand-written adjoint of the library.

forward() calls sps_loglike_grad once and keeps the gradient it returns;
backward() scales that cached gradient by the incoming one.  The per-SSP
products are recomputed inside the library rather than stored."""
from __future__ import annotations

import torch


class SpsLoglike(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta, sps, mag_obs, sigma, mask, gal_idx=None, mode="approx", prec="fp32"):
        ll, g = sps.loglike_grad(theta.detach().contiguous(), mag_obs, sigma, mask,
                                 gal_idx=gal_idx, mode=mode, prec=prec, grad=True)
        ctx.save_for_backward(g)
        return ll

    @staticmethod
    def backward(ctx, grad_ll):
        (g,) = ctx.saved_tensors
        return grad_ll[:, None] * g, None, None, None, None, None, None, None


def loglike(theta, sps, mag_obs, sigma, mask, gal_idx=None, mode="approx", prec="fp32"):
    return SpsLoglike.apply(theta, sps, mag_obs, sigma, mask, gal_idx, mode, prec)
