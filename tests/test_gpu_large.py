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
