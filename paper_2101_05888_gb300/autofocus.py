"""Differentiable backprojection and sharpness-based autofocus.

SAS platform motion has to be estimated from the data itself (Sec. I, item 2;
Sec. II-D).  This module exposes the backprojection as a function of per-ping
position offsets dp (added to the navigation) whose backward pass is the
library's hand-written adjoint kernel, and a small autofocus loop that
maximises the image sharpness S = sum|I|^4 / (sum|I|^2)^2 over dp.

Everything numeric runs in libsas kernels: the forward image
(sas_backproject_2d/3d), S and dS/dI* (sas_sharpness) and dS/d(dp)
(sas_backproject_adjoint with an offset-gradient output, image tiles
recomputed rather than stored).  PyTorch only holds the tensors.
"""
from __future__ import annotations

import torch

import paper_2101_05888_gb300 as sas


class BackprojectOffsets(torch.autograd.Function):
    """image = B(dp): forward backprojection with per-ping offsets dp [P,3]
    (float64, device).  Backward maps dL/dimage to dL/d(dp) with the adjoint
    kernel.  PyTorch hands a real loss's complex gradient to backward as
    dL/dRe + i dL/dIm = 2 dL/dI*, which is halved here because the kernel
    takes dL/dI*."""

    @staticmethod
    def forward(ctx, offsets, geom, grid, interp):
        geom.set_offsets(offsets.detach().contiguous())
        image = geom.backproject(grid, interp)
        ctx.geom, ctx.grid, ctx.interp = geom, grid, interp
        ctx.save_for_backward(offsets)
        return image

    @staticmethod
    def backward(ctx, grad_image):
        (offsets,) = ctx.saved_tensors
        geom = ctx.geom
        geom.set_offsets(offsets.detach().contiguous())
        G = (0.5 * grad_image).contiguous()
        grad = torch.empty((geom.P, 3), dtype=torch.float64, device=grad_image.device)
        sas.sas_backproject_adjoint(geom.h, ctx.grid, ctx.interp, G, None, grad)
        return grad, None, None, None


def backproject_offsets(offsets, geom, grid, interp=None):
    return BackprojectOffsets.apply(offsets, geom, grid, interp or sas.kaiser())


def sharpness_and_grad(image):
    """S (float) and dS/dI* (complex64, same shape) from the library kernel."""
    out = torch.zeros(3, dtype=torch.float64, device=image.device)
    g = torch.empty_like(image)
    sas.sas_sharpness(image, image.numel(), out, g)
    return out, g


def offset_gradient(geom, grid, interp, offsets):
    """S(dp) and dS/d(dp) [P,3] for the current echo."""
    geom.set_offsets(offsets)
    image = geom.backproject(grid, interp)
    out, g = sharpness_and_grad(image)
    grad = torch.empty((geom.P, 3), dtype=torch.float64, device=image.device)
    sas.sas_backproject_adjoint(geom.h, grid, interp, g, None, grad)
    return out, grad


def autofocus(geom, grid, steps: int = 20, step_m: float = 1e-3, interp=None, offsets=None, beta=0.9,
              shrink=0.5):
    """Gradient ascent on the sharpness over per-ping offsets.

    Each step moves dp by ``step_m`` metres (rms over the P x 3 entries) along
    a momentum-averaged, normalised gradient.  A step that lowers S is undone
    and the step length multiplied by ``shrink``, so the returned history of S
    (one value per step, starting from the initial offsets) never decreases.
    Returns (offsets, history of S)."""
    interp = interp or sas.kaiser()
    dev = torch.device("cuda")
    dp = torch.zeros((geom.P, 3), dtype=torch.float64, device=dev) if offsets is None else offsets.clone()
    out, grad = offset_gradient(geom, grid, interp, dp)
    best_s, best_dp, best_grad = float(out[0].item()), dp, grad
    mom = torch.zeros_like(dp)
    hist = [best_s]
    step = step_m
    for _ in range(steps):
        mom = beta * mom + (1.0 - beta) * best_grad
        rms = torch.sqrt(torch.mean(mom * mom)).clamp_min(1e-300)
        trial = best_dp + step * mom / rms
        out, grad = offset_gradient(geom, grid, interp, trial)
        s = float(out[0].item())
        if s >= best_s:
            best_s, best_dp, best_grad = s, trial, grad
        else:
            step *= shrink
            mom = torch.zeros_like(dp)
        hist.append(best_s)
    geom.set_offsets(best_dp)
    return best_dp, hist
