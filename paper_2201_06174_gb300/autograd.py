"""torch.autograd.Function over the C ABI: gradients of the consolidated saliency map with
respect to the input volume, the 3 combination weights and the per-direction weights of the
center-surround window (so that those weights can be fitted to an interpreter's template).

The forward runs sal_saliency with the given weights and keeps its features E and raw maps S3
(6 volumes); the backward runs the adjoint of each step on them -- sal_combine_backward,
sal_center_surround_backward, sal_local_spectra_project_backward (which recomputes the local
spectra brick by brick; no spectrum is stored) -- so no step of the forward runs twice.  The
min-max bounds of the forward pass are held constant.
"""
from __future__ import annotations

import torch

from . import sal as _sal


class SaliencyFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, V, W, alpha, engine):
        engine.set_alpha(alpha.detach().cpu().numpy())
        S = torch.empty(engine.shape, dtype=torch.float32, device=engine.device)
        E = torch.empty((3,) + tuple(engine.shape), dtype=torch.float32, device=engine.device)
        S3 = torch.empty_like(E)
        _sal.sal_saliency(engine.h, V.contiguous(), None, W.contiguous(), S, S3, E)
        ctx.save_for_backward(V, W, alpha, E, S3)
        ctx.engine = engine
        return S

    @staticmethod
    def backward(ctx, gS):
        V, W, alpha, E, S3 = ctx.saved_tensors
        eng = ctx.engine
        eng.set_alpha(alpha.detach().cpu().numpy())
        gW = torch.empty(3, dtype=torch.float32, device=V.device)
        galpha = torch.empty_like(alpha)
        gS3 = torch.empty_like(S3)
        _sal.sal_combine_backward(eng.h, S3, W.contiguous(), gS.contiguous(), gS3, gW)
        gE = torch.empty_like(E)
        _sal.sal_center_surround_backward(eng.h, E, gS3, gE, galpha)
        gV = None
        if ctx.needs_input_grad[0]:
            gV = torch.empty_like(V)
            _sal.sal_local_spectra_project_backward(eng.h, V.contiguous(), gE, gV)
        return gV, gW, galpha, None


def saliency(V: torch.Tensor, W: torch.Tensor, alpha: torch.Tensor, engine: "_sal.Saliency") -> torch.Tensor:
    """Differentiable consolidated saliency map S(V; W, alpha) on the engine's volume shape."""
    return SaliencyFunction.apply(V, W, alpha, engine)
