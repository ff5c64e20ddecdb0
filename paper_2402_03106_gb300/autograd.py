"""Differentiable transient rendering: a torch.autograd.Function around
darts_render (forward) and darts_adjoint (path-replay backward).

The forward pass renders the histogram h(sigma_s, sigma_a, g) with the
sampling's seed; the backward pass re-traces an independent set of paths
(seed `adjoint_seed`) and returns d(sum_b grad_h[b] h_b)/d(sigma_s, sigma_a,
g) with every sampling density held fixed.  Using an independent seed keeps
the product (h - target) * dh/dtheta of an L2 loss free of the correlation
bias a shared seed would introduce.
"""
from __future__ import annotations

import dataclasses
from typing import Optional

import torch

from . import capi, scenes as S


def _with_medium(scene: S.Scene, sigma_s, sigma_a, g) -> S.Scene:
    m = dataclasses.replace(scene.medium, sigma_s=float(sigma_s), sigma_a=float(sigma_a), g=float(g))
    return dataclasses.replace(scene, medium=m)


class DartsRender(torch.autograd.Function):
    @staticmethod
    def forward(ctx, sigma_s, sigma_a, g, scene, sampling, adjoint_seed, dctx):
        sc = _with_medium(scene, sigma_s.item(), sigma_a.item(), g.item())
        h = dctx.render(sc, sampling)
        ctx.scene = sc
        ctx.sampling = dataclasses.replace(sampling, seed=int(adjoint_seed),
                                           flags=sampling.flags & ~S.FLAG_REBUILD_TABLE)
        ctx.dctx = dctx
        ctx.param_meta = (sigma_s.dtype, sigma_s.device)
        return h

    @staticmethod
    def backward(ctx, grad_h):
        g3 = ctx.dctx.adjoint(ctx.scene, ctx.sampling, grad_h)
        dtype, device = ctx.param_meta
        g3 = g3.to(device=device, dtype=dtype)
        return g3[0], g3[1], g3[2], None, None, None, None


def render(sigma_s: torch.Tensor, sigma_a: torch.Tensor, g: torch.Tensor, scene: S.Scene,
           sampling: S.Sampling, adjoint_seed: Optional[int] = None,
           dctx: Optional[capi.Context] = None) -> torch.Tensor:
    """Differentiable histogram [n_bins] (float64, on the context's device).
    sigma_s, sigma_a, g: scalar tensors (requires_grad as needed)."""
    if dctx is None:
        dctx = capi.Context(torch.cuda.current_device())
    if adjoint_seed is None:
        adjoint_seed = (int(sampling.seed) * 0x9E3779B97F4A7C15 + 0x632BE59BD9B4E019) & ((1 << 64) - 1)
    return DartsRender.apply(sigma_s, sigma_a, g, scene, sampling, adjoint_seed, dctx)
