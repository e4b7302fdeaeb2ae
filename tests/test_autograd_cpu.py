"""The Eq. 1 surrogate EpsAdjoint, without a GPU: its fused library call
(eps_vjp_surrogate) is replaced by the FP64 oracle (eps_hat, J^T w and the
sum of eps_hat * w over the J-support voxels, of the same inputs), so that
the wrapper's own plumbing is what is tested, and the surrogate's
definition is pinned against Eq. 1 by finite differences.

- S(C) equals scale * sum over the J-support voxels (Ex/Ey planes
  k0+1 .. k0+nk, Ez planes k0 .. k0+nk) of eps_hat * Re(sum_l E_F,l E_A,l),
  with the product unconjugated;
- S.backward() leaves the call's dJ/dC, times the incoming gradient, in
  C.grad, and the fields get none;
- the gradient of S is Eq. 1: torch.autograd.gradcheck compares it with
  central differences of S itself;
- no wavelengths give S = 0 and a zero gradient."""

import numpy as np
import pytest
import torch

from oracle import epschain_oracle as orc
from paper_2505_03352_gb300 import autograd as ag
from paper_2505_03352_gb300 import epschain as eb


def _oracle_problem(p):
    return orc.Problem(mx=p.mx, my=p.my, nz=p.nz, radius=p.radius, beta=p.beta, eta=p.eta,
                       eps_core=p.eps_core, eps_clad=p.eps_clad, sub=p.sub, slab_nk=p.slab_nk,
                       slab_k0=p.slab_k0, bc=p.bc)


def _support_mask(o):
    # the voxels whose eps_hat depends on C (z rules of Sec. 3's extrusion)
    m = np.zeros((3, o.nx, o.ny, o.nz), dtype=bool)
    k0, nk = o.k0, o.slab_nk
    m[0:2, :, :, k0 + 1:k0 + nk + 1] = True
    m[2, :, :, k0:k0 + nk + 1] = True
    return m


@pytest.fixture
def oracle_call(monkeypatch):
    """eps_vjp_surrogate(prob, C, EF, EA, scale, eps_out) answered by the
    oracle."""
    calls = []

    def fused(prob, C, EF, EA, scale=-2.0, eps_out=None, **kw):
        o = _oracle_problem(prob)
        Cn = C.detach().numpy().astype(np.float64)
        w = np.zeros((3, o.nx, o.ny, o.nz))
        for ef, ea in zip(EF, EA):
            w += (ef.numpy() * ea.numpy()).real
        calls.append(len(EF))
        e = orc.eps_hat(o, Cn)
        S = torch.tensor(float(np.sum((e * scale * w)[_support_mask(o)])), dtype=torch.float64)
        g = torch.from_numpy(orc.vjp_real(o, Cn, scale * w))
        return (g, torch.from_numpy(e), S) if eps_out is True else (g, S)

    monkeypatch.setattr(ag, "eps_vjp_surrogate", fused)
    return calls


P = eb.Problem(mx=10, my=8, nz=7, radius=1.5, beta=4.0, slab_nk=3)


def _inputs(seed, n_lambda=2):
    rng = np.random.default_rng(seed)
    C = torch.from_numpy(rng.random((P.mx, P.my)))
    shape = (3, P.nx, P.ny, P.nz)
    EF = [torch.from_numpy(rng.standard_normal(shape) + 1j * rng.standard_normal(shape))
          for _ in range(n_lambda)]
    EA = [torch.from_numpy(rng.standard_normal(shape) + 1j * rng.standard_normal(shape))
          for _ in range(n_lambda)]
    return C, EF, EA


def test_surrogate_value_and_gradient(oracle_call):
    C, EF, EA = _inputs(1)
    C.requires_grad_(True)
    S, eps = ag.eps_adjoint(C, P, EF, EA, scale=-2.0, with_eps=True)
    assert S.dtype == torch.float64 and not eps.requires_grad
    o = _oracle_problem(P)
    e = orc.eps_hat(o, C.detach().numpy())
    np.testing.assert_array_equal(eps.numpy(), e)
    w = sum((ef.numpy() * ea.numpy()).real for ef, ea in zip(EF, EA))
    assert S.item() == pytest.approx(-2.0 * float(np.sum((e * w)[_support_mask(o)])), rel=1e-12)
    # the cladding voxels hold eps_clad whatever C is: summing over every
    # voxel instead changes S by a constant only
    full = -2.0 * float(np.sum(e * w))
    e2 = orc.eps_hat(o, C.detach().numpy() * 0.5)
    S2 = ag.eps_adjoint(C.detach() * 0.5, P, EF, EA)
    full2 = -2.0 * float(np.sum(e2 * w))
    assert (full - S.item()) == pytest.approx(full2 - S2.item(), rel=1e-10)
    (3.0 * S).backward()
    ref = orc.vjp_fields(o, C.detach().numpy(), [x.numpy() for x in EF], [x.numpy() for x in EA])
    np.testing.assert_allclose(C.grad.numpy(), 3.0 * ref, rtol=1e-12, atol=1e-14 * np.abs(ref).max())
    assert oracle_call == [2, 2]


def test_surrogate_gradient_is_eq1_by_central_differences(oracle_call):
    C, EF, EA = _inputs(2)
    C.requires_grad_(True)
    assert torch.autograd.gradcheck(lambda c: ag.eps_adjoint(c, P, EF, EA), (C,), eps=1e-6,
                                    atol=1e-7, rtol=1e-5)


def test_no_wavelengths_give_a_zero_surrogate(oracle_call):
    C, _, _ = _inputs(3)
    C.requires_grad_(True)
    S = ag.eps_adjoint(C, P, [], [])
    S.backward()
    assert S.item() == 0.0 and torch.count_nonzero(C.grad).item() == 0
