"""torch.autograd wrapper of the permittivity chain.

EpsChain.apply(C, prob) returns eps_hat [3, nx, ny, nz] (eps_forward); its
backward is the vector-Jacobian product of Sec. 3 for the incoming real
cotangent (eps_vjp_real).  Only C is saved for the backward pass: the
filtered density and projection are recomputed there, so no activation of
the chain is kept alive between forward and backward.

For the optimiser loop of the paper, where the cotangent is the Eq. 1 field
product, adjoint_gradient() makes one fused call that returns eps_hat and
dJ/dC together.
"""

from __future__ import annotations

import torch

from .epschain import (EPS_FIELD_C64, Morph, Problem, eps_forward, eps_forward_morph, eps_vjp,
                       eps_vjp_real, eps_vjp_real_morph)


class EpsChain(torch.autograd.Function):
    @staticmethod
    def forward(ctx, C, prob: Problem):
        if C.dtype != torch.float32:
            raise TypeError("C must be float32")
        C = C.contiguous()
        eps = eps_forward(prob, C)
        ctx.prob = prob
        ctx.save_for_backward(C)
        return eps

    @staticmethod
    def backward(ctx, grad_eps):
        (C,) = ctx.saved_tensors
        G = grad_eps.contiguous().to(torch.float32)
        return eps_vjp_real(ctx.prob, C, G), None


def eps_chain(C, prob: Problem):
    """Differentiable eps_hat(C) (see EpsChain)."""
    return EpsChain.apply(C, prob)


def adjoint_gradient(prob: Problem, C, EF, EA, scale: float = -2.0, field_type: int = EPS_FIELD_C64,
                     field_scales=None, ws=None, stream=None):
    """Eq. 1 in one fused call: returns (eps_hat, dJ/dC) for forward fields EF
    and adjoint fields EA (lists, one tensor per wavelength)."""
    dJdC, eps = eps_vjp(prob, C, EF, EA, scale=scale, eps_out=True, field_type=field_type,
                        field_scales=field_scales, ws=ws, stream=stream)
    return eps, dJdC


class EpsChainMorph(torch.autograd.Function):
    """eps_hat(C) through the chain with morphological filtering (Eq. 3-6);
    backward is eps_vjp_real_morph, which recomputes every map from C."""

    @staticmethod
    def forward(ctx, C, prob: Problem, morph: Morph):
        if C.dtype != torch.float32:
            raise TypeError("C must be float32")
        C = C.contiguous()
        eps = eps_forward_morph(prob, morph, C)
        ctx.prob = prob
        ctx.morph = morph
        ctx.save_for_backward(C)
        return eps

    @staticmethod
    def backward(ctx, grad_eps):
        (C,) = ctx.saved_tensors
        G = grad_eps.contiguous().to(torch.float32)
        return eps_vjp_real_morph(ctx.prob, ctx.morph, C, G), None, None


def eps_chain_morph(C, prob: Problem, morph: Morph):
    """Differentiable eps_hat(C) with morphology (see EpsChainMorph)."""
    return EpsChainMorph.apply(C, prob, morph)
