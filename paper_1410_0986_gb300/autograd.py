"""Differentiable Born product: forward y = J x, backward x_bar = J^T y_bar.

The misfit gradient with respect to the chromophore maps (Section 5, the gradient
-(d mu/d p)^T H^T (y - H mu) of the reconstruction) is J^T r; here it comes from the
hand-written adjoint kernel (hydot_born_apply_T), with the fields held as
non-differentiable context.
"""
from __future__ import annotations

import torch


class BornApply(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, context, phi_src, phi_det, lam0: int, nlam: int):
        ctx.context = context
        ctx.lam = (lam0, nlam)
        ctx.save_for_backward(phi_src, phi_det)
        return context.born_apply(phi_src, phi_det, lam0, nlam, x.contiguous())

    @staticmethod
    def backward(ctx, gy):
        phi_src, phi_det = ctx.saved_tensors
        lam0, nlam = ctx.lam
        g = ctx.context.born_apply_T(phi_src, phi_det, lam0, nlam, gy.contiguous())
        return g, None, None, None, None, None


def born_apply(x, context, phi_src, phi_det, lam0: int, nlam: int):
    """y = J x over the wavelength slice, differentiable in x."""
    return BornApply.apply(x, context, phi_src, phi_det, lam0, nlam)
