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

import ctypes

from .epschain import (EPS_FIELD_C64, Morph, Problem, _check, _field_ptrs, _need, _ptr, _scales,
                       _stream, _workspace, eps_forward, eps_forward_morph, eps_vjp, eps_vjp_real,
                       eps_vjp_real_morph, eps_vjp_surrogate, lib)


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
        # eps_hat is not differentiable: without this, autograd would fill a
        # zero gradient of eps_hat's size (hundreds of MB) for every backward
        ctx.set_materialize_grads(False)
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
        if grad_S is None:
            return None, None, None, None, None, None
        return grad_S.to(dJdC.dtype) * dJdC, None, None, None, None, None


def eps_adjoint(C, prob: Problem, EF, EA, scale: float = -2.0, with_eps: bool = False):
    """The Eq. 1 surrogate S(C) (see EpsAdjoint), a float64 0-d tensor;
    S.backward() leaves dJ/dC in C.grad.  With with_eps, returns (S, eps_hat)
    from the same fused call (eps_hat is what the next field solve needs)."""
    return EpsAdjoint.apply(C, prob, list(EF), list(EA), scale, with_eps)


class AdjointSurrogate:
    """EpsAdjoint for fields that stay fixed over many calls (the inner loop
    of an optimisation between two field solves): the fused call's field
    pointers, scales and workspace are checked and marshalled once, and each
    call passes only C.  surr(C) returns S (or (S, eps_hat) with with_eps),
    differentiable in C exactly as eps_adjoint's.  The tensors given here
    must stay alive and unchanged in shape while the object is used; calls
    of one object share its workspace, so they must not overlap on
    different streams."""

    def __init__(self, prob: Problem, EF, EA, scale: float = -2.0, with_eps: bool = False,
                 field_type: int = EPS_FIELD_C64, field_scales=None):
        dev = EF[0].device if len(EF) else torch.device("cuda", torch.cuda.current_device())
        self.prob = prob
        self.with_eps = with_eps
        self._dev = dev
        self._nl, self._ef, self._ea = _field_ptrs(prob, EF, EA, field_type, dev)
        self._fs = _scales(field_scales, self._nl)
        self._ws = _workspace(prob, self._nl, None, dev)
        self._keep = (list(EF), list(EA))
        self._p = prob.c_struct()
        self._field_type = field_type
        self._scale = float(scale)
        self._fn = lib().eps_vjp_surrogate

    def call(self, C):
        """One fused call: returns (dJdC, eps_hat or None, S)."""
        _need(C, (self.prob.mx, self.prob.my), torch.float32, "C", self._dev)
        dJdC = torch.empty((self.prob.mx, self.prob.my), dtype=torch.float32, device=self._dev)
        S = torch.empty((), dtype=torch.float64, device=self._dev)
        eps = (torch.empty((3, self.prob.nx, self.prob.ny, self.prob.nz), dtype=torch.float32,
                           device=self._dev) if self.with_eps else None)
        _check(self._fn(ctypes.byref(self._p), _ptr(C), self._nl, self._field_type, self._ef,
                        self._ea, self._fs, self._scale, _ptr(dJdC), _ptr(eps), _ptr(S),
                        _ptr(self._ws), self._ws.numel(), _stream(None)),
               "eps_vjp_surrogate")
        return dJdC, eps, S

    def __call__(self, C):
        return _PreparedAdjoint.apply(C, self)


class _PreparedAdjoint(torch.autograd.Function):
    """EpsAdjoint through an AdjointSurrogate's prepared call."""

    @staticmethod
    def forward(ctx, C, surr: AdjointSurrogate):
        ctx.set_materialize_grads(False)   # no zero gradient of eps_hat (see EpsAdjoint)
        dJdC, eps, S = surr.call(C.contiguous())
        ctx.save_for_backward(dJdC)
        if eps is not None:
            ctx.mark_non_differentiable(eps)
            return S, eps
        return S

    @staticmethod
    def backward(ctx, grad_S, *unused):
        (dJdC,) = ctx.saved_tensors
        if grad_S is None:
            return None, None
        return grad_S.to(dJdC.dtype) * dJdC, None


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
