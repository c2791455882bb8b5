"""torch.autograd.Function over gsp_render_fwd / gsp_render_bwd (L1 photometric loss).

forward returns the L1 loss computed in the library; backward replays the
composite back to front in the library, with the L1 sign map formed on the
device, and optionally accumulates the edge score in the same pass.
"""
from __future__ import annotations

import torch

from .api import Renderer


class GaussianRenderL1(torch.autograd.Function):
    @staticmethod
    def forward(ctx, means, log_scales, quats, opacity_logits, sh, renderer: Renderer, targets, edge=None,
                score=None, pos_grad=None):
        # the parameter tensors are the renderer's GaussianSet storage
        out = renderer.forward(targets=targets, edge=None, score=None, want_loss=True)
        ctx.renderer = renderer
        ctx.fwd = out
        ctx.targets = targets
        ctx.edge = edge
        ctx.score = score
        ctx.pos_grad = pos_grad  # (sum, count) of the gradient-threshold masking, or None
        return out["loss"].reshape(())

    @staticmethod
    def backward(ctx, grad_loss):
        r = ctx.renderer
        grads = r.backward(ctx.fwd, targets=ctx.targets, edge=ctx.edge, score=ctx.score, pos_grad=ctx.pos_grad)
        # the library's adjoint is that of L itself; scale by the incoming gradient
        g = grad_loss.reshape(1)
        out = []
        for name in ("means", "log_scales", "quats", "opacity_logits", "sh"):
            out.append(grads[name].mul_(g))
        return (*out, None, None, None, None, None)
