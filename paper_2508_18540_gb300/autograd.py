"""torch.autograd bindings of the differentiable G2LF / V2LF path.

The forward runs lf_build_mpi_* and lf_composite; the backward runs
lf_composite_backward and lf_build_mpi_backward_* (liblf kernels). The
integer structure of the forward (culling, chunks, plane depths, footprints,
tile lists, nearest indices) is held fixed and receives no gradient.

The renderer's workspace carries the forward's structure into the backward,
so a renderer must not render again between a forward and its backward;
that is checked.
"""
from __future__ import annotations

import torch

from . import api


class _RenderGaussians(torch.autograd.Function):
    @staticmethod
    def forward(ctx, renderer, means, scales, quats, opacity, rgb):
        g = api.DeviceGaussians(means.detach().contiguous(), scales.detach().contiguous(),
                                quats.detach().contiguous(), opacity.detach().contiguous(), rgb.detach().contiguous())
        renderer.render(g)
        ctx.renderer, ctx.g, ctx.generation = renderer, g, renderer.generation
        return renderer.out.clone()

    @staticmethod
    def backward(ctx, dviews):
        r = ctx.renderer
        if r.generation != ctx.generation:
            raise RuntimeError("the renderer rendered again before this backward; its workspace no longer "
                               "holds this forward's structure")
        grads, _ = r.backward(ctx.g, dviews.contiguous().float())
        return None, grads.dmeans, grads.dscales, grads.dquats, grads.dopacity, grads.drgb


class _RenderVoxels(torch.autograd.Function):
    @staticmethod
    def forward(ctx, renderer, prims, density8, rgb):
        v = api.DeviceVoxels(prims.ijk, prims.level, density8.detach().contiguous(), rgb.detach().contiguous(),
                             prims.origin, prims.base_size)
        renderer.render(v)
        ctx.renderer, ctx.v, ctx.generation = renderer, v, renderer.generation
        return renderer.out.clone()

    @staticmethod
    def backward(ctx, dviews):
        r = ctx.renderer
        if r.generation != ctx.generation:
            raise RuntimeError("the renderer rendered again before this backward; its workspace no longer "
                               "holds this forward's structure")
        grads, _ = r.backward(ctx.v, dviews.contiguous().float())
        return None, None, grads.ddensity8, grads.drgb


def render_gaussians(renderer: api.LightFieldRenderer, means, scales, quats, opacity, rgb) -> torch.Tensor:
    """Differentiable light-field render of 3D Gaussians: views [V][Ny][Nx][4]."""
    return _RenderGaussians.apply(renderer, means, scales, quats, opacity, rgb)


def render_voxels(renderer: api.LightFieldRenderer, prims: api.DeviceVoxels, density8, rgb) -> torch.Tensor:
    """Differentiable light-field render of sparse voxels (densities and colours)."""
    return _RenderVoxels.apply(renderer, prims, density8, rgb)
