"""Differentiation form: the dirty image as a differentiable function of the
complex gains (torch.autograd), and a gradient gain solve.

EpicImageFn.apply(gains, volt, plan) -> image [C][N][N] float64.  Forward is
epic_image with the given gains; backward is epic_image_backward (the
hand-written adjoint kernel).  Gradients follow torch's complex convention
(2 dL/dconj(g)).
"""
from __future__ import annotations

import torch


class EpicImageFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, gains, volt, plan):
        plan.set_gains_device(gains.detach().contiguous())
        img = plan.image(volt)
        ctx.save_for_backward(gains.detach(), volt)
        ctx.plan = plan
        return img

    @staticmethod
    def backward(ctx, grad_img):
        gains, volt = ctx.saved_tensors
        plan = ctx.plan
        plan.set_gains_device(gains.contiguous())
        grad = plan.image_backward(volt, grad_img.contiguous())
        return grad, None, None


def chi2(image, model):
    """L = sum (I - M)^2 over channels and pixels."""
    return ((image - model) ** 2).sum()


def solve_gains(plan, volt, model, g0, steps=200, lr=0.02, decay=1.0, callback=None):
    """Minimise chi2(I(g), M) over the complex gains with Adam (learning rate
    multiplied by `decay` after every step), the gradient coming from the
    adjoint kernel.  Returns the final gains (detached)."""
    g = g0.detach().clone().requires_grad_(True)
    opt = torch.optim.Adam([g], lr=lr)
    sched = torch.optim.lr_scheduler.ExponentialLR(opt, gamma=decay)
    for it in range(steps):
        opt.zero_grad(set_to_none=True)
        loss = chi2(EpicImageFn.apply(g, volt, plan), model)
        loss.backward()
        opt.step()
        sched.step()
        if callback is not None:
            callback(it, loss.detach(), g.detach())
    return g.detach()
