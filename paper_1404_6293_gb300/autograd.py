"""Differentiable rendering through the rasterizer's shading.

``render(rasterizer, scene, color, normal, light)`` returns the RGBA image
and the depth|ID key buffer; gradients flow to the per-vertex colours,
normals and the light direction.  Visibility is held fixed by the forward
pass's key buffer, so coverage stays exact integer arithmetic and only the
shading (Gouraud, or the Lambert shader of Listing 1 in the Piko paper) is
differentiated; the backward pass is the library's own kernel
(piko_raster_backward), with no autograd of PyTorch operations in between.
"""
from __future__ import annotations

import dataclasses
from typing import Optional

import torch

from .raster import DeviceScene, Rasterizer


class _RasterShade(torch.autograd.Function):
    @staticmethod
    def forward(ctx, color, normal, light, rasterizer: Rasterizer, scene: DeviceScene):
        ds = dataclasses.replace(scene, color=color, normal=normal, light_dir=light)
        fb = rasterizer.forward(ds)
        ctx.rasterizer, ctx.scene, ctx.fb = rasterizer, ds, fb
        ctx.needs = (color is not None and ctx.needs_input_grad[0],
                     normal is not None and ctx.needs_input_grad[1],
                     light is not None and ctx.needs_input_grad[2])
        ctx.mark_non_differentiable(fb.key)
        return fb.rgba, fb.key

    @staticmethod
    def backward(ctx, g_rgba, g_key):
        ds = ctx.scene
        need_c, need_n, need_l = ctx.needs
        dc = torch.zeros_like(ds.color) if need_c else None
        dn = torch.zeros_like(ds.normal) if need_n else None
        dl = torch.zeros_like(ds.light_dir) if need_l else None
        if g_rgba is not None and (need_c or need_n or need_l):
            ctx.rasterizer.backward(ds, ctx.fb, g_rgba.contiguous(), dc, dn, dl)
        return dc, dn, dl, None, None


def render(rasterizer: Rasterizer, scene: DeviceScene, color: Optional[torch.Tensor] = None,
           normal: Optional[torch.Tensor] = None, light: Optional[torch.Tensor] = None):
    """Rasterizes ``scene`` with the given (optionally differentiable)
    attributes; tensors left as None fall back to the scene's own.
    Returns (rgba float32 [H,W,4], key int64 [H,W])."""
    c = scene.color if color is None else color
    n = scene.normal if normal is None else normal
    l = scene.light_dir if light is None else light
    return _RasterShade.apply(c, n, l, rasterizer, scene)
