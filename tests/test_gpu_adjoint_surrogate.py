"""EpsAdjoint, the Eq. 1 surrogate, on the GPU.

- Small case, both stencil launch forms' code paths for S: its gradient is
  the fused eps_vjp call's dJ/dC bit for bit and the oracle's within 1e-4,
  and its value (summed by the library in FP64) is the oracle's sum of
  eps_hat * w over the J-support voxels.
- The differentiation form at full size: 2000 x 2000 controls, 1000 x 1000 x
  32, three wavelengths of seeded complex64 E_F and E_A, through
  torch.autograd (S = eps_adjoint(C, ...); S.backward()), in the launch
  configuration the benchmark times; C.grad against the oracle on windows,
  S against an FP64 sum over the device arrays.
"""

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


def _support_sum(o, e, w):
    """sum of e * w over the voxels whose eps_hat depends on C: Ex and Ey
    planes k0+1 .. k0+nk, Ez planes k0 .. k0+nk"""
    k0, nk = o.k0, o.slab_nk
    return (float(np.sum(e[0:2, :, :, k0 + 1:k0 + nk + 1] * w[0:2, :, :, k0 + 1:k0 + nk + 1]))
            + float(np.sum(e[2, :, :, k0:k0 + nk + 1] * w[2, :, :, k0:k0 + nk + 1])))


# 64 x 48: one wave (each tile waits for the contraction and adds to S);
# 1200 x 1040 (600 x 520 Yee columns, 1275 tiles): several waves (the seeds
# kernel adds to S, four columns per thread); 1202 x 1042 (an odd column
# count): the seeds kernel's one-column-per-thread form
@pytest.mark.parametrize("mx,my", [(64, 48), (1200, 1040), (1202, 1042)],
                         ids=["one_wave", "multi_wave", "multi_wave_odd_columns"])
def test_adjoint_surrogate_value_and_gradient(mx, my):
    torch, ec, ag = _mods()
    p = ec.Problem(mx=mx, my=my, nz=16, radius=3.0, beta=8.0)
    o = orc.Problem(mx=mx, my=my, nz=16, radius=3.0, beta=8.0)
    Cn = np.random.default_rng(21).random((mx, my), dtype=np.float32)
    shape = (3, p.nx, p.ny, p.nz)
    EFn = [synth.complex_field(shape, 22 + l) for l in range(2)]
    EAn = [synth.complex_field(shape, 32 + l) for l in range(2)]
    C = torch.from_numpy(Cn).cuda()
    EF = [torch.from_numpy(e).cuda() for e in EFn]
    EA = [torch.from_numpy(e).cuda() for e in EAn]
    ref_g, ref_e = ec.eps_vjp(p, C, EF, EA, eps_out=True)
    Cg = C.clone().requires_grad_(True)
    S, eps = ag.eps_adjoint(Cg, p, EF, EA, with_eps=True)
    S.backward()
    torch.testing.assert_close(Cg.grad, ref_g, rtol=0, atol=0)
    torch.testing.assert_close(eps, ref_e, rtol=0, atol=0)
    w = -2.0 * sum((ef.astype(np.complex128) * ea).real for ef, ea in zip(EFn, EAn))
    e_or = orc.eps_hat(o, Cn)
    ref_S = _support_sum(o, e_or, w)
    mag = _support_sum(o, e_or, np.abs(w))
    # eps_hat within 1e-5 of the oracle and FP32 column sums: S within 1e-5
    # of the sum of the magnitudes of its terms
    assert abs(S.item() - ref_S) <= 1e-5 * mag, (S.item(), ref_S, mag)
    if mx <= 64:
        ref = orc.vjp_fields(o, Cn, EFn, EAn)
        assert np.max(np.abs(Cg.grad.cpu().numpy() - ref)) / np.max(np.abs(ref)) <= 1e-4


def test_prepared_surrogate_equals_the_functional_form():
    # AdjointSurrogate (fields marshalled once) against eps_adjoint: the same
    # S, eps_hat and gradient bit for bit, on two calls in a row with C
    # changed in place between them (an optimiser step)
    torch, ec, ag = _mods()
    p = ec.Problem(mx=200, my=168, nz=16, radius=3.0, beta=8.0)
    shape = (3, p.nx, p.ny, p.nz)
    EF = [torch.from_numpy(synth.complex_field(shape, 42 + l)).cuda() for l in range(3)]
    EA = [torch.from_numpy(synth.complex_field(shape, 52 + l)).cuda() for l in range(3)]
    C = torch.from_numpy(np.random.default_rng(23).random((200, 168), dtype=np.float32)).cuda()
    surr = ag.AdjointSurrogate(p, EF, EA, with_eps=True)
    Cp = C.clone().requires_grad_(True)
    for step in range(2):
        Cp.grad = None
        S, eps = surr(Cp)
        S.backward()
        Cf = Cp.detach().clone().requires_grad_(True)
        Sf, epsf = ag.eps_adjoint(Cf, p, EF, EA, with_eps=True)
        Sf.backward()
        assert S.item() == Sf.item()
        torch.testing.assert_close(eps, epsf, rtol=0, atol=0)
        torch.testing.assert_close(Cp.grad, Cf.grad, rtol=0, atol=0)
        with torch.no_grad():
            Cp.sub_(1e-3 * torch.sign(Cp.grad))


def test_differentiation_form_at_full_size():
    # cfg3 through autograd, three wavelengths: C.grad on five windows against
    # the oracle (the chain is local; see tests/test_gpu_large.py), S against
    # an FP64 reduction of the device's own eps_hat and fields
    torch, ec, ag = _mods()
    from tests.test_gpu_large import _device_fields, window_check_device
    w = synth.WORKLOADS[3]
    C = synth.controls(w)
    p = ec.Problem(mx=w.mx, my=w.my, nz=w.nz, radius=w.radius, beta=w.beta)
    EF = _device_fields((3, w.nx, w.ny, w.nz), 3, 2030)
    EA = _device_fields((3, w.nx, w.ny, w.nz), 3, 3030)
    Cg = torch.from_numpy(C).cuda().requires_grad_(True)
    S, eps = ag.eps_adjoint(Cg, p, EF, EA, with_eps=True)
    S.backward()
    ec.eps_sync_status()
    windows = [(0, 0), (1000, 1000), (w.mx, w.my), (0, w.my), (517, 1733)]
    worst_e, worst_g = window_check_device(w, C, EF, EA, eps.cpu().numpy(),
                                           Cg.grad.cpu().numpy(), windows)
    assert worst_e <= 1e-5, worst_e
    assert worst_g <= 1e-4, worst_g
    k0, nk = p.k0, p.slab_nk
    ref_S = torch.zeros((), dtype=torch.float64, device="cuda")
    mag = torch.zeros((), dtype=torch.float64, device="cuda")
    e64 = eps.double()
    for ef, ea in zip(EF, EA):
        wl = -2.0 * (ef.real.double() * ea.real.double() - ef.imag.double() * ea.imag.double())
        ref_S += (e64[0:2, :, :, k0 + 1:k0 + nk + 1] * wl[0:2, :, :, k0 + 1:k0 + nk + 1]).sum()
        ref_S += (e64[2, :, :, k0:k0 + nk + 1] * wl[2, :, :, k0:k0 + nk + 1]).sum()
        mag += (e64[0:2, :, :, k0 + 1:k0 + nk + 1] * wl[0:2, :, :, k0 + 1:k0 + nk + 1]).abs().sum()
        mag += (e64[2, :, :, k0:k0 + nk + 1] * wl[2, :, :, k0:k0 + nk + 1]).abs().sum()
        del wl
    assert abs(S.item() - ref_S.item()) <= 1e-6 * mag.item(), (S.item(), ref_S.item())
    del EF, EA, eps
    torch.cuda.empty_cache()
