"""Differentiable Lambertian shading: a torch.autograd.Function whose forward and
backward are the library's grtShadeLambert / grtShadeLambertBackward kernels.

The forward traces the primary hits (closest hit on the geometry), shades them and,
in "store" mode, keeps the hit records and visibility for the adjoint; in
"recompute" mode it drops them and the adjoint traces again (21 bytes per pixel
saved). Positions are differentiated at interior hits; the geometry must have been
built (or refit) from the same positions before the forward pass.
"""
from __future__ import annotations

import torch

from . import grtShadeLambert, grtShadeLambertBackward, grtTraceClosest
from .objects import new_hits


class LambertRenderer:
    """Rays, geometry and mesh indices shared by forward and backward passes."""

    def __init__(self, ctx, geometry, indices: torch.Tensor, rays: torch.Tensor, store: bool = True, opts=None):
        self.ctx = ctx
        self.geometry = geometry
        self.indices = indices
        self.rays = rays
        self.n = rays.shape[0]
        self.store = store
        self.opts = opts


class LambertShade(torch.autograd.Function):
    @staticmethod
    def forward(fctx, colours: torch.Tensor, light: torch.Tensor, positions: torch.Tensor, R: LambertRenderer):
        colours = colours.contiguous()
        light = light.contiguous()
        positions = positions.contiguous()
        stream = torch.cuda.current_stream().cuda_stream
        hits = new_hits(R.n)
        grtTraceClosest(R.ctx.handle, None, R.geometry.handle, R.rays, R.n, hits, None, R.opts, stream)
        image = torch.empty((R.n, 3), dtype=torch.float32, device=colours.device)
        vis = torch.empty(R.n, dtype=torch.uint8, device=colours.device) if R.store else None
        grtShadeLambert(R.ctx.handle, R.geometry.handle, R.rays, hits, R.n, R.indices, positions, colours, light,
                        image, vis, R.opts, stream)
        # the hit records and visibility of THIS forward stay with its autograd node, so
        # several forwards through one renderer each get their own backward
        fctx.R = R
        fctx.hits, fctx.vis = (hits, vis) if R.store else (None, None)
        fctx.save_for_backward(colours, light, positions)
        return image

    @staticmethod
    def backward(fctx, grad_image: torch.Tensor):
        colours, light, positions = fctx.saved_tensors
        R = fctx.R
        gc = torch.zeros_like(colours)
        gl = torch.zeros_like(light)
        gp = torch.zeros_like(positions)
        grtShadeLambertBackward(R.ctx.handle, R.geometry.handle, R.rays, fctx.hits, fctx.vis, R.n, R.indices, positions,
                                colours, light, grad_image.contiguous(), gc, gl, gp, R.opts,
                                torch.cuda.current_stream().cuda_stream)
        return gc, gl, gp, None


def lambert_shade(colours, light, positions, renderer: LambertRenderer) -> torch.Tensor:
    """Differentiable image (n, 3) of the renderer's rays."""
    return LambertShade.apply(colours, light, positions, renderer)
