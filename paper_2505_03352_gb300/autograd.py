"""torch.autograd wrapper of the permittivity chain.

EpsChain.apply(C, prob) returns eps_hat [3, nx, ny, nz] (eps_forward); its
backward is the vector-Jacobian product of Sec. 3 for the incoming real
cotangent (eps_vjp_real).  Only C is saved for the backward pass: the
filtered density and projection are recomputed there, so no activation of
the chain is kept alive between forward and backward.

For the optimiser loop of the paper, where the cotangent is the Eq. 1 field
product, adjoint_gradient() makes one fused call that returns eps_hat and
dJ/dC together, and EpsAdjoint exposes the fused call to autograd as a
scalar (computed by the library) whose gradient is Eq. 1.
"""

from __future__ import annotations

import torch

from .epschain import (EPS_FIELD_C64, Morph, Problem, eps_forward, eps_forward_morph, eps_vjp,
                       eps_vjp_real, eps_vjp_real_morph, eps_vjp_surrogate)


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


class EpsAdjoint(torch.autograd.Function):
    """Scalar surrogate of the adjoint method (Eq. 1):

        S(C) = sum over the J-support voxels of eps_hat(C) * w,
        w = scale Re(sum_l E_F,l * E_A,l)   (unconjugated, held fixed),

    so that dS/dC = J^T w is Eq. 1's dJ/dC (scale = -2).  The J-support
    voxels are those where eps_hat depends on C; the cladding voxels would
    only add a constant.  The forward makes one eps_vjp_surrogate call,
    which computes dJ/dC, S (FP64, summed on the device) and, if asked,
    eps_hat in the same pass; it saves dJ/dC, and the backward scales it by
    the incoming gradient.  The fields are complex64 lists (one tensor per
    wavelength) and are not differentiated; eps_hat, when returned, is not
    differentiable either."""

    @staticmethod
    def forward(ctx, C, prob: Problem, EF, EA, scale: float = -2.0, with_eps: bool = False):
        C = C.contiguous()
        if with_eps:
            dJdC, eps, S = eps_vjp_surrogate(prob, C, EF, EA, scale=scale, eps_out=True)
            ctx.mark_non_differentiable(eps)
        else:
            dJdC, S = eps_vjp_surrogate(prob, C, EF, EA, scale=scale)
        ctx.save_for_backward(dJdC)
        return (S, eps) if with_eps else S

    @staticmethod
    def backward(ctx, grad_S, *unused):
        (dJdC,) = ctx.saved_tensors
        return grad_S.to(dJdC.dtype) * dJdC, None, None, None, None, None


def eps_adjoint(C, prob: Problem, EF, EA, scale: float = -2.0, with_eps: bool = False):
    """The Eq. 1 surrogate S(C) (see EpsAdjoint), a float64 0-d tensor;
    S.backward() leaves dJ/dC in C.grad.  With with_eps, returns (S, eps_hat)
    from the same fused call (eps_hat is what the next field solve needs)."""
    return EpsAdjoint.apply(C, prob, list(EF), list(EA), scale, with_eps)


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
