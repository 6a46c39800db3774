"""torch.autograd binding of the fused NLL + gradient pass.

`nll(model, events, theta)` returns the NLL as a 0-dim CUDA tensor whose
backward is grad_output times the analytic gradient computed in the same event
pass (ipa_nll_grad): one kernel pass gives both, so an optimiser step costs one
pass.  `nll_joint(model, events, seg_off, joint, theta)` does the same for
simultaneous fits over categories (ipa_nll_grad_joint): one NLL per fit,
theta (n_fits x n_joint).  Event columns are constants of the graph (no
gradient flows to them).
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


class JointNLLFunction(torch.autograd.Function):
    """forward: the joint NLL of every fit (ipa_nll_grad_joint); backward:
    grad_output[i] * dNLL_i/dtheta_i."""

    @staticmethod
    def forward(ctx, theta: torch.Tensor, model, events: dict, seg_off: torch.Tensor, joint) -> torch.Tensor:
        out = api.ipa_nll_grad_joint(model, events, seg_off, joint, theta.detach().contiguous())
        ctx.save_for_backward(out[:, 1:])
        ctx.shape = theta.shape
        return out[:, 0]

    @staticmethod
    def backward(ctx, grad_output: torch.Tensor):
        (g,) = ctx.saved_tensors
        return (grad_output[:, None] * g).reshape(ctx.shape), None, None, None, None


def nll_joint(model, events: dict, seg_off: torch.Tensor, joint, theta: torch.Tensor) -> torch.Tensor:
    """Differentiable joint NLL per fit (a vector of n_fits) of simultaneous fits
    at theta (float64 CUDA tensor, n_fits x n_joint)."""
    return JointNLLFunction.apply(theta, model, events, seg_off, joint)

