"""Full-size workloads in the launch configuration the benchmark uses,
checked against the FP64 oracle on windows.

The chain is local: eps_hat at a cell depends on C within R + 4 subpixels,
and dJ/dC at a control on C and the fields within about 2R + 8 subpixels.
So the oracle, run on a window grown by that margin (or cut at the region
edge, where it applies the same boundary rule), reproduces the full-size
result exactly in the window's interior.
"""

import numpy as np
import pytest

from oracle import epschain_oracle as orc
from paper_2505_03352_gb300 import synth

pytestmark = pytest.mark.gpu

EPS_TOL = 1e-5
GRAD_TOL = 1e-4


def window_check(w, C, EF, EA, eps_gpu, g_gpu, windows, half=48):
    margin = int(2 * np.ceil(w.radius)) + 8
    margin += margin % 2
    worst_e = worst_g = 0.0
    for (ca, cb) in windows:
        a0 = max(0, ca - half) // 2 * 2
        b0 = max(0, cb - half) // 2 * 2
        a1 = min(w.mx, a0 + 2 * half)
        b1 = min(w.my, b0 + 2 * half)
        wa0, wb0 = max(0, a0 - margin), max(0, b0 - margin)
        wa1, wb1 = min(w.mx, a1 + margin), min(w.my, b1 + margin)
        o = orc.Problem(mx=wa1 - wa0, my=wb1 - wb0, nz=w.nz, radius=w.radius, beta=w.beta)
        Cw = C[wa0:wa1, wb0:wb1]
        EFw = [e[:, wa0 // 2:wa1 // 2, wb0 // 2:wb1 // 2, :] for e in EF]
        EAw = [e[:, wa0 // 2:wa1 // 2, wb0 // 2:wb1 // 2, :] for e in EA]
        ref_e = orc.eps_hat(o, Cw)
        ref_g = orc.vjp_fields(o, Cw, EFw, EAw)
        # interior of the window, in window coordinates
        ia0, ib0, ia1, ib1 = a0 - wa0, b0 - wb0, a1 - wa0, b1 - wb0
        re = ref_e[:, ia0 // 2:ia1 // 2, ib0 // 2:ib1 // 2, :]
        ge = eps_gpu[:, a0 // 2:a1 // 2, b0 // 2:b1 // 2, :]
        rg = ref_g[ia0:ia1, ib0:ib1]
        gg = g_gpu[a0:a1, b0:b1]
        worst_e = max(worst_e, float(np.max(np.abs(ge - re) / np.abs(re))))
        worst_g = max(worst_g, float(np.max(np.abs(gg - rg)) / np.max(np.abs(rg))))
    return worst_e, worst_g


def test_cfg3_three_wavelengths_windows():
    import torch

    import paper_2505_03352_gb300 as ec
    w = synth.WORKLOADS[3]
    C = synth.controls(w)
    EF, EA = synth.fields(w)
    p = ec.Problem(mx=w.mx, my=w.my, nz=w.nz, radius=w.radius, beta=w.beta)
    g, e = ec.eps_vjp(p, torch.from_numpy(C).cuda(), [torch.from_numpy(x).cuda() for x in EF],
                      [torch.from_numpy(x).cuda() for x in EA], eps_out=True)
    ec.eps_sync_status()
    g, e = g.cpu().numpy(), e.cpu().numpy()
    windows = [(0, 0), (1000, 1000), (w.mx, w.my), (0, w.my), (517, 1733)]
    worst_e, worst_g = window_check(w, C, EF, EA, e, g, windows)
    assert worst_e <= EPS_TOL, worst_e
    assert worst_g <= GRAD_TOL, worst_g


def _device_fields(shape, n, seed):
    import torch
    g = torch.Generator(device="cuda")
    out = []
    for l in range(n):
        g.manual_seed(seed + l)
        out.append(torch.randn(tuple(shape) + (2,), generator=g, device="cuda")
                   .view(torch.complex64)[..., 0].contiguous())
    return out


def window_check_device(w, C, EF, EA, eps_gpu, g_gpu, windows, half=48, prob=None):
    """window_check for fields held on the device: only each window's slice
    of the fields is copied to the host for the oracle."""
    margin = int(2 * np.ceil(w.radius)) + 8
    margin += margin % 2
    worst_e = worst_g = 0.0
    for (ca, cb) in windows:
        a0 = max(0, ca - half) // 2 * 2
        b0 = max(0, cb - half) // 2 * 2
        a1 = min(w.mx, a0 + 2 * half)
        b1 = min(w.my, b0 + 2 * half)
        wa0, wb0 = max(0, a0 - margin), max(0, b0 - margin)
        wa1, wb1 = min(w.mx, a1 + margin), min(w.my, b1 + margin)
        o = orc.Problem(mx=wa1 - wa0, my=wb1 - wb0, nz=w.nz, radius=w.radius, beta=w.beta)
        sl = (slice(None), slice(wa0 // 2, wa1 // 2), slice(wb0 // 2, wb1 // 2), slice(None))
        Cw = C[wa0:wa1, wb0:wb1]
        ref_g = orc.vjp_fields(o, Cw, [e[sl].cpu().numpy() for e in EF],
                               [e[sl].cpu().numpy() for e in EA])
        ia0, ib0, ia1, ib1 = a0 - wa0, b0 - wb0, a1 - wa0, b1 - wb0
        rg = ref_g[ia0:ia1, ib0:ib1]
        gg = g_gpu[a0:a1, b0:b1]
        worst_g = max(worst_g, float(np.max(np.abs(gg - rg)) / np.max(np.abs(rg))))
        if eps_gpu is not None:
            re = orc.eps_hat(o, Cw)[:, ia0 // 2:ia1 // 2, ib0 // 2:ib1 // 2, :]
            ge = eps_gpu[:, a0 // 2:a1 // 2, b0 // 2:b1 // 2, :]
            worst_e = max(worst_e, float(np.max(np.abs(ge - re) / np.abs(re))))
    return worst_e, worst_g


def test_cfg5_eight_wavelengths_at_full_size():
    # 3000 x 3000 controls, 1500 x 1500 x 32, eight wavelengths (27.6 GB of
    # complex64 fields on the device), in the bench's launch configuration;
    # the FP32 path within the oracle tolerance, BF16 and FP16 fields within
    # about 1.5 times their measured quantisation error
    import torch

    import paper_2505_03352_gb300 as ec
    w = synth.WORKLOADS[5]
    C = synth.controls(w)
    p = ec.Problem(mx=w.mx, my=w.my, nz=w.nz, radius=w.radius, beta=w.beta)
    EF = _device_fields((3, w.nx, w.ny, w.nz), 8, 2050)
    EA = _device_fields((3, w.nx, w.ny, w.nz), 8, 3050)
    Cd = torch.from_numpy(C).cuda()
    g, e = ec.eps_vjp(p, Cd, EF, EA, eps_out=True)
    ec.eps_sync_status()
    g, e = g.cpu().numpy(), e.cpu().numpy()
    windows = [(0, 0), (1500, 1500), (w.mx, w.my), (0, w.my), (2210, 377)]
    worst_e, worst_g = window_check_device(w, C, EF, EA, e, g, windows)
    assert worst_e <= EPS_TOL, worst_e
    assert worst_g <= GRAD_TOL, worst_g
    print(f"cfg5 FP32: eps_hat {worst_e:.3e}, dJ/dC {worst_g:.3e}")
    # quantisation error of the packed formats on these windows, measured on
    # a GB300: BF16 6.29e-3, FP16 4.10e-4 of the largest value; the gates sit
    # about 1.5 times above (the inputs and the kernels are deterministic)
    for ft, bound in ((ec.EPS_FIELD_BF16X2_SCALED, 9.5e-3), (ec.EPS_FIELD_F16X2_SCALED, 6.2e-4)):
        PF = [ec.eps_field_pack(p, ft, x) for x in EF]
        PA = [ec.eps_field_pack(p, ft, x) for x in EA]
        gq = ec.eps_vjp(p, Cd, PF, PA, field_type=ft)
        ec.eps_sync_status()
        _, worst_q = window_check_device(w, C, EF, EA, None, gq.cpu().numpy(), windows[:3])
        print(f"cfg5 field type {ft}: dJ/dC {worst_q:.3e}")
        assert worst_q <= bound, (ft, worst_q)
        del PF, PA
    del EF, EA
    torch.cuda.empty_cache()


def test_cfg4_batch_at_full_size():
    # the 64-region batch (sides 64 .. 1014, radii 2 .. 8) in one batched
    # call: the smallest, a median and the largest region checked on windows
    import torch

    import paper_2505_03352_gb300 as ec
    regs = synth.batched_regions()
    probs, Cs, EFs, EAs, Ch = [], [], [], [], []
    for r, rw in enumerate(regs):
        probs.append(ec.Problem(mx=rw.mx, my=rw.my, nz=rw.nz, radius=rw.radius, beta=rw.beta))
        C = synth.soi_layout(rw.mx, rw.my, 1004 * 1000 + r)
        Ch.append(C)
        Cs.append(torch.from_numpy(C).cuda())
        EFs.append(_device_fields((3, rw.nx, rw.ny, rw.nz), 1, 2040 * 1000 + r))
        EAs.append(_device_fields((3, rw.nx, rw.ny, rw.nz), 1, 3040 * 1000 + r))
    bv = ec.BatchedVjp(probs, Cs, EFs, EAs)
    G, E = bv()
    ec.eps_sync_status()
    sides = [rw.mx for rw in regs]
    for k in (int(np.argmin(sides)), int(np.argsort(sides)[len(sides) // 2]), int(np.argmax(sides))):
        rw = regs[k]
        windows = [(0, 0), (rw.mx // 2, rw.my // 2), (rw.mx, rw.my)]
        worst_e, worst_g = window_check_device(rw, Ch[k], EFs[k], EAs[k], E[k].cpu().numpy(),
                                               G[k].cpu().numpy(), windows)
        assert worst_e <= EPS_TOL, (k, worst_e)
        assert worst_g <= GRAD_TOL, (k, worst_g)
