"""eps_vjp_static, the entry point that allocates nothing, against eps_vjp.

This file is collected last on purpose: if it fails, a run that stops at the
first failure has already run every other test.  It calls the C ABI directly
(ctypes), twice in a row on the same inputs, and compares with eps_vjp given
a workspace, within the parity tolerances of the other GPU tests.
"""

import ctypes

import numpy as np
import pytest

from paper_2505_03352_gb300 import synth

pytestmark = pytest.mark.gpu

EPS_TOL = 1e-5
GRAD_TOL = 1e-4


def _setup():
    import torch

    import paper_2505_03352_gb300 as ec
    from paper_2505_03352_gb300 import epschain as eb
    L = eb.lib()
    L.eps_vjp_static.restype = ctypes.c_int
    L.eps_vjp_static.argtypes = [ctypes.POINTER(eb.eps_problem_t), ctypes.c_void_p, ctypes.c_int32,
                                 ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                 ctypes.c_float, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    return torch, ec, eb, L


def _static_call(torch, eb, L, prob, C, EF, EA, dJdC, eps):
    p = prob.c_struct()
    ef = (ctypes.c_void_p * 1)(EF.data_ptr())
    ea = (ctypes.c_void_p * 1)(EA.data_ptr())
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return L.eps_vjp_static(ctypes.byref(p), C.data_ptr(), 1, eb.EPS_FIELD_C64, ef, ea, None,
                            -2.0, dJdC.data_ptr(), eps.data_ptr(), stream)


def test_static_scratch_matches_workspace_version_twice():
    torch, ec, eb, L = _setup()
    w = synth.WORKLOADS[2]
    prob = ec.Problem(mx=w.mx, my=w.my, nz=w.nz, radius=w.radius, beta=w.beta)
    C = torch.from_numpy(synth.controls(w)).cuda()
    EF, EA = synth.fields(w)
    EFd = torch.from_numpy(EF[0]).cuda()
    EAd = torch.from_numpy(EA[0]).cuda()
    ref_g, ref_e = ec.eps_vjp(prob, C, [EFd], [EAd], eps_out=True)
    ec.eps_sync_status()
    ref_g, ref_e = ref_g.cpu().numpy(), ref_e.cpu().numpy()
    scale = np.max(np.abs(ref_g))
    for _ in range(2):
        dJdC = torch.full((w.mx, w.my), float("nan"), device="cuda")
        eps = torch.full((3, w.nx, w.ny, w.nz), float("nan"), device="cuda")
        st = _static_call(torch, eb, L, prob, C, EFd, EAd, dJdC, eps)
        assert st == eb.EPS_OK, eb.STATUS_NAMES.get(st, st)
        ec.eps_sync_status()
        g, e = dJdC.cpu().numpy(), eps.cpu().numpy()
        assert np.max(np.abs(g - ref_g)) / scale <= GRAD_TOL
        assert np.max(np.abs(e - ref_e) / np.abs(ref_e)) <= EPS_TOL


def test_static_scratch_rejects_problems_beyond_its_size():
    torch, ec, eb, L = _setup()
    prob = ec.Problem(mx=1200, my=1200, nz=24, radius=6.0, beta=16.0)
    need = ec.eps_workspace_size(prob)
    assert need > 16 * 1024 * 1024
    C = torch.zeros((prob.mx, prob.my), device="cuda")
    F = torch.zeros((3, prob.nx, prob.ny, prob.nz), dtype=torch.complex64, device="cuda")
    dJdC = torch.zeros((prob.mx, prob.my), device="cuda")
    eps = torch.zeros((3, prob.nx, prob.ny, prob.nz), device="cuda")
    st = _static_call(torch, eb, L, prob, C, F, F, dJdC, eps)
    assert st == 3   # EPS_ERR_WORKSPACE, returned before any launch
