"""torch.autograd.Function of the chain: gradients against the FP64 oracle,
against the C-ABI VJP, and against finite differences of the GPU forward."""

import numpy as np
import pytest

from oracle import epschain_oracle as orc
from paper_2505_03352_gb300 import synth

pytestmark = pytest.mark.gpu


def _mods():
    import torch

    import paper_2505_03352_gb300 as ec
    from paper_2505_03352_gb300 import autograd as ag
    return torch, ec, ag


@pytest.mark.parametrize("bc", [0, 1])
def test_backward_matches_oracle_vjp(bc):
    torch, ec, ag = _mods()
    mx, my, nz = 70, 98, 16
    p = ec.Problem(mx=mx, my=my, nz=nz, radius=3.0, beta=8.0, bc=bc)
    o = orc.Problem(mx=mx, my=my, nz=nz, radius=3.0, beta=8.0, bc=bc)
    rng = np.random.default_rng(11)
    Cn = rng.random((mx, my), dtype=np.float32)
    Gn = rng.standard_normal((3, p.nx, p.ny, nz)).astype(np.float32)
    C = torch.from_numpy(Cn).cuda().requires_grad_(True)
    eps = ag.eps_chain(C, p)
    (eps * torch.from_numpy(Gn).cuda()).sum().backward()
    got = C.grad.cpu().numpy()
    ref = orc.vjp_real(o, Cn, Gn)
    assert np.max(np.abs(got - ref)) / np.max(np.abs(ref)) <= 1e-4
    np.testing.assert_allclose(eps.detach().cpu().numpy(), orc.eps_hat(o, Cn), rtol=1e-5)


def test_backward_equals_c_abi_vjp_real():
    torch, ec, ag = _mods()
    p = ec.Problem(mx=64, my=64, nz=16, radius=3.0, beta=16.0)
    C = torch.rand((64, 64), device="cuda").requires_grad_(True)
    G = torch.randn((3, 32, 32, 16), device="cuda")
    ag.eps_chain(C, p).backward(G)
    ref = ec.eps_vjp_real(p, C.detach(), G)
    torch.testing.assert_close(C.grad, ref, rtol=0, atol=0)


def test_directional_finite_difference_of_the_gpu_forward():
    torch, ec, ag = _mods()
    w = synth.WORKLOADS[1]
    p = ec.Problem(mx=w.mx, my=w.my, nz=w.nz, radius=w.radius, beta=w.beta)
    C0 = torch.from_numpy(synth.controls(w)).cuda()
    G = torch.randn((3, p.nx, p.ny, p.nz), device="cuda", generator=torch.Generator("cuda").manual_seed(3))
    v = torch.randn(C0.shape, device="cuda", generator=torch.Generator("cuda").manual_seed(4))
    C = C0.clone().requires_grad_(True)
    (ag.eps_chain(C, p) * G).sum().backward()
    dd = float((C.grad * v).sum())
    h = 1e-3
    with torch.no_grad():
        jp = float((ec.eps_forward(p, (C0 + h * v).contiguous()).double() * G.double()).sum())
        jm = float((ec.eps_forward(p, (C0 - h * v).contiguous()).double() * G.double()).sum())
    fd = (jp - jm) / (2 * h)
    assert abs(fd - dd) <= 1e-2 * abs(dd)


def test_adjoint_gradient_is_the_fused_call():
    torch, ec, ag = _mods()
    w = synth.WORKLOADS[1]
    p = ec.Problem(mx=w.mx, my=w.my, nz=w.nz, radius=w.radius, beta=w.beta)
    o = orc.Problem(mx=w.mx, my=w.my, nz=w.nz, radius=w.radius, beta=w.beta)
    Cn = synth.controls(w)
    EF, EA = synth.fields(w)
    eps, g = ag.adjoint_gradient(p, torch.from_numpy(Cn).cuda(), [torch.from_numpy(e).cuda() for e in EF],
                                 [torch.from_numpy(e).cuda() for e in EA])
    ref = orc.vjp_fields(o, Cn, EF, EA)
    assert np.max(np.abs(g.cpu().numpy() - ref)) / np.max(np.abs(ref)) <= 1e-4

