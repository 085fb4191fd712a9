"""torch.autograd.Function over the batched fill and its hand-written adjoint.

    out = guidefill_fill(rgba, labels, mag, phi, mu, eps=3.0, c=0.05)
    loss = 0.5 * ((out - gt) ** 2).sum(); loss.backward()

rgba [B,H,W,4] float32, labels [B,H,W] uint8, guidance as magnitude mag [B,H,W]
and angle phi [B,H,W] (g = mag (cos phi, sin phi)), mu a 0-d tensor.
Gradients flow to rgba (the known colours), phi and mu; the shell schedule,
the stall steps and each ghost sample's tap set are held fixed (piecewise
constant).  Both passes run in libguidefill.so; the forward keeps only the shell
map, the stall bitmap, the guide field and its output for the backward.
"""
from __future__ import annotations

import torch

from . import context


class GuidefillFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, rgba, labels, mag, phi, mu, eps, c):
        g = context(rgba.device.index)
        B = rgba.shape[0]
        muf = float(mu)
        guides = [g.guide_from_angle(labels[i], mag[i], phi[i]) for i in range(B)]
        res = g.fill_batched([rgba[i] for i in range(B)], [labels[i] for i in range(B)], guides, eps=eps, mu=muf,
                             c=c, stall=True)
        out = torch.stack([r.rgba for r in res])
        ctx.res = res
        ctx.guides = guides
        ctx.eps, ctx.mu, ctx.c = eps, muf, c
        ctx.mu_device = mu.device if torch.is_tensor(mu) else None
        return out

    @staticmethod
    def backward(ctx, grad_out):
        g = context(grad_out.device.index)
        B = grad_out.shape[0]
        gi, gp, gmu = g.fill_backward(ctx.res, ctx.guides, [grad_out[i] for i in range(B)], eps=ctx.eps,
                                      mu=ctx.mu, c=ctx.c)
        grad_rgba = torch.stack(gi)
        grad_phi = torch.stack(gp)
        grad_mu = gmu.sum()
        if ctx.mu_device is not None:
            grad_mu = grad_mu.to(ctx.mu_device)
        return grad_rgba, None, None, grad_phi, grad_mu, None, None


def guidefill_fill(rgba, labels, mag, phi, mu, eps=3.0, c=0.05):
    if not torch.is_tensor(mu):
        mu = torch.tensor(float(mu))
    return GuidefillFunction.apply(rgba, labels, mag, phi, mu, eps, c)
