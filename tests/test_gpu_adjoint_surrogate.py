"""EpsAdjoint, the Eq. 1 surrogate, on the GPU: its gradient is the fused
eps_vjp call's dJ/dC bit for bit and the oracle's within 1e-4, and its value
is the sum over that call's eps_hat."""

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


def test_adjoint_surrogate_backward_is_the_fused_call():
    # S = -2 sum eps_hat Re(sum_l E_F E_A): its gradient is the fused call's
    # dJ/dC bit for bit, its value a sum over that call's eps_hat, and the
    # gradient matches the oracle's Eq. 1
    torch, ec, ag = _mods()
    p = ec.Problem(mx=64, my=48, nz=16, radius=3.0, beta=8.0)
    o = orc.Problem(mx=64, my=48, nz=16, radius=3.0, beta=8.0)
    Cn = np.random.default_rng(21).random((64, 48), dtype=np.float32)
    shape = (3, p.nx, p.ny, p.nz)
    EFn = [synth.complex_field(shape, 22 + l) for l in range(2)]
    EAn = [synth.complex_field(shape, 32 + l) for l in range(2)]
    C = torch.from_numpy(Cn).cuda()
    EF = [torch.from_numpy(e).cuda() for e in EFn]
    EA = [torch.from_numpy(e).cuda() for e in EAn]
    ref_g, ref_e = ec.eps_vjp(p, C, EF, EA, eps_out=True)
    Cg = C.clone().requires_grad_(True)
    S = ag.eps_adjoint(Cg, p, EF, EA)
    S.backward()
    torch.testing.assert_close(Cg.grad, ref_g, rtol=0, atol=0)
    terms = ref_e.cpu().numpy().astype(np.float64) * sum((ef * ea).real for ef, ea in zip(EFn, EAn))
    assert abs(S.item() - (-2.0) * terms.sum()) <= 1e-5 * 2.0 * np.abs(terms).sum()
    ref = orc.vjp_fields(o, Cn, EFn, EAn)
    assert np.max(np.abs(Cg.grad.cpu().numpy() - ref)) / np.max(np.abs(ref)) <= 1e-4
