"""Differentiable rendering: the forward render and its hand-written
adjoint (osog_render_keep / osog_render_backward_kept) as a
torch.autograd.Function.

The paper's pipeline is differentiable end to end so that dI/dTheta drives
inverse rendering (Sec. III.C, Sec. IV.B).  Here the particle tensor and the
optics scalars (defocus, DIC shear length, shear angle and bias) are the
differentiable inputs; gradients come from libosog's adjoint kernels, not
from autograd tracing.
"""
from __future__ import annotations

import torch

from ._lib import OsogError
from .render import Renderer

INVALID_ARG = 1  # osog_render_backward_kept: no kept forward state matches

OPTICS_PARAMS = ("defocus", "shear_px", "shear_angle", "bias_phase")


def optics_with(optics: dict, params) -> dict:
    """Copy of `optics` with the four differentiable scalars replaced."""
    o = dict(optics)
    vals = params.detach().double().cpu().tolist() if torch.is_tensor(params) else list(params)
    for k, v in zip(OPTICS_PARAMS, vals):
        o[k] = float(v)
    return o


class RenderFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, soa, optics_params, renderer: Renderer, optics: dict):
        o = optics_with(optics, optics_params)
        soa_c = soa.detach().contiguous()
        if any(ctx.needs_input_grad[:2]):
            # the forward intermediates stay in a workspace of this call's
            # own, so the adjoint need not recompute them
            img, ws = renderer.render_keep(soa_c, None, o)
        else:
            img, ws = renderer.render(soa_c, None, o), None
        ctx.save_for_backward(soa_c)
        ctx.renderer, ctx.optics, ctx.ws = renderer, o, ws
        ctx.params_meta = (optics_params.dtype, optics_params.device)
        return img

    @staticmethod
    def backward(ctx, grad_image):
        (soa,) = ctx.saved_tensors
        g = grad_image.contiguous().float()
        gsoa = gopt = None
        if ctx.ws is not None:
            try:
                gsoa, gopt = ctx.renderer.backward_kept(soa, None, ctx.optics, g, ctx.ws)
            except OsogError as e:
                # the plan remembers the states of its last 64 workspaces; an
                # older one was dropped, so the adjoint recomputes the forward
                if e.code != INVALID_ARG:
                    raise
            ctx.ws = None  # consumed: a second backward recomputes the forward
        if gsoa is None:
            gsoa, gopt = ctx.renderer.backward(soa, None, ctx.optics, g)
        dtype, device = ctx.params_meta
        return gsoa, gopt.to(device=device, dtype=dtype), None, None


def render(soa: torch.Tensor, optics: dict, renderer: Renderer,
           optics_params: torch.Tensor | None = None) -> torch.Tensor:
    """Differentiable (K, H, W) render of one scene.  `optics_params` holds
    (defocus, shear_px, shear_angle, bias_phase); when None the values of
    `optics` are used and receive no gradient."""
    if optics_params is None:
        optics_params = torch.tensor([float(optics[k]) for k in OPTICS_PARAMS])
    return RenderFunction.apply(soa, optics_params, renderer, optics)
