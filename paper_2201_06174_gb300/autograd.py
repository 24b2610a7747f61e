"""torch.autograd.Function over the C ABI: gradients of the consolidated saliency map with
respect to the input volume, the 3 combination weights and the per-direction weights of the
center-surround window (so that those weights can be fitted to an interpreter's template).

The forward runs sal_saliency with the given weights; the backward runs
sal_saliency_backward, which recomputes the local spectra brick by brick (nothing but V, W
and alpha is saved).  The min-max bounds of the forward pass are held constant.
"""
from __future__ import annotations

import torch

from . import sal as _sal


class SaliencyFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, V, W, alpha, engine):
        engine.set_alpha(alpha.detach().cpu().numpy())
        S = torch.empty(engine.shape, dtype=torch.float32, device=engine.device)
        _sal.sal_saliency(engine.h, V.contiguous(), None, W.contiguous(), S)
        ctx.save_for_backward(V, W, alpha)
        ctx.engine = engine
        return S

    @staticmethod
    def backward(ctx, gS):
        V, W, alpha = ctx.saved_tensors
        eng = ctx.engine
        eng.set_alpha(alpha.detach().cpu().numpy())
        gV = torch.empty_like(V) if ctx.needs_input_grad[0] else None
        gW = torch.empty(3, dtype=torch.float32, device=V.device)
        galpha = torch.empty_like(alpha)
        _sal.sal_saliency_backward(eng.h, V.contiguous(), W.contiguous(), gS.contiguous(), gV, gW, galpha)
        return gV, gW, galpha, None


def saliency(V: torch.Tensor, W: torch.Tensor, alpha: torch.Tensor, engine: "_sal.Saliency") -> torch.Tensor:
    """Differentiable consolidated saliency map S(V; W, alpha) on the engine's volume shape."""
    return SaliencyFunction.apply(V, W, alpha, engine)
