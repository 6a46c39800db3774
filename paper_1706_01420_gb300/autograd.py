"""torch.autograd binding of the fused NLL + gradient pass.

`nll(model, events, theta)` returns the NLL as a 0-dim CUDA tensor whose
backward is grad_output times the analytic gradient computed in the same event
pass (ipa_nll_grad): one kernel pass gives both, so an optimiser step costs one
pass.  Event columns are constants of the graph (no gradient flows to them).
"""
from __future__ import annotations

import torch

from . import api


class NLLFunction(torch.autograd.Function):
    """forward: NLL = -sum w log P (ipa_nll_grad); backward: grad_output * dNLL/dtheta."""

    @staticmethod
    def forward(ctx, theta: torch.Tensor, model, events: dict) -> torch.Tensor:
        out = api.ipa_nll_grad(model, events, theta.detach().contiguous())
        ctx.save_for_backward(out[1:])
        return out[0]

    @staticmethod
    def backward(ctx, grad_output: torch.Tensor):
        (g,) = ctx.saved_tensors
        return grad_output * g, None, None


def nll(model, events: dict, theta: torch.Tensor) -> torch.Tensor:
    """Differentiable NLL of `events` at `theta` (float64 CUDA tensor of n_par values)."""
    return NLLFunction.apply(theta, model, events)
