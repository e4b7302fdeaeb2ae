"""On-device optimiser iteration (Eq. 10-15) against the FP64 optimiser
oracle.  Both sides get the same seeded synthetic gradient G (no oracle
input comes from the CUDA path); the design's gray count is taken by the
GPU from its own VJP workspace and by the oracle from its own forward.
Gray decisions near the threshold may differ between FP32 and FP64: the
counts must agree up to the number of subpixels whose rho (1 - rho) lies
within 1e-4 (relative) of gray_tol (1 - gray_tol)."""

import numpy as np
import pytest

from oracle import epschain_oracle as orc
from oracle import morph_oracle as mo
from oracle import optimizer_oracle as oo
from paper_2505_03352_gb300 import synth

pytestmark = pytest.mark.gpu


def _ec():
    import paper_2505_03352_gb300 as ec
    return ec


def to_dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).cuda()


def near_threshold(rho, tol):
    q = rho * (1 - rho)
    thr = tol * (1 - tol)
    return int(np.count_nonzero(np.abs(q - thr) <= 1e-4 * thr))


def run_loop(n_steps, morph=None, real=False, mx=64, my=64, nz=16, radius=3.0, binary=False):
    import dataclasses
    import torch
    ec = _ec()
    params = dict(lr=0.01, n_iter=12, beta_min=4.0, beta_max0=40.0, gray_tol=0.05)
    opt, oopt = ec.OptParams(**params), oo.OptParams(**params)
    C = synth.soi_layout(mx, my, 5100, sigma=3.0).astype(np.float64)
    if binary:
        C = (C > 0.5).astype(np.float64)
    p_gpu = ec.Problem(mx=mx, my=my, nz=nz, radius=radius, beta=1.0)
    o_base = orc.Problem(mx=mx, my=my, nz=nz, radius=radius, beta=1.0)
    Cd = to_dev(C)
    Md = torch.zeros_like(Cd)
    Vd = torch.zeros_like(Cd)
    M = np.zeros_like(C)
    V = np.zeros_like(C)
    state = ec.eps_opt_init(opt)
    s_ref = oo.init_state(oopt)
    st = ec.read_opt_state(state)
    assert st["step"] == 0 and st["gray_acc"] == 0 and st["ticket"] == 0
    assert abs(st["beta"] - s_ref.beta) <= 1e-6 * s_ref.beta
    shape = (3, mx // 2, my // 2, nz)
    EF = [torch.from_numpy(synth.complex_field(shape, 5101)).cuda()]
    EA = [torch.from_numpy(synth.complex_field(shape, 5102)).cuda()]
    results = []
    for it in range(n_steps):
        beta_gpu = ec.read_opt_state(state)["beta"]
        p = dataclasses.replace(p_gpu, beta=beta_gpu)
        o = dataclasses.replace(o_base, beta=s_ref.beta)
        # the VJP that evaluates the design at this beta (its dJ/dC is not used:
        # both sides step with the same synthetic gradient)
        if morph is None:
            ws = torch.empty(ec.eps_workspace_size(p), dtype=torch.uint8, device="cuda")
            if real:
                Gr = to_dev(np.random.default_rng(it).standard_normal(shape))
                ec.eps_vjp_real(p, Cd, Gr, ws=ws)
            else:
                ec.eps_vjp(p, Cd, EF, EA, ws=ws)
            rho = orc.forward(o, C)["rho"]
        else:
            ws = torch.empty(ec.eps_morph_workspace_size(p, morph), dtype=torch.uint8, device="cuda")
            ec.eps_vjp_morph(p, morph, Cd, EF, EA, ws=ws)
            om = mo.Morph(alpha=morph.alpha, radius=morph.radius, ops=morph.ops)
            rho = mo.forward_morph(o, om, C)["rho"]
        G = np.random.default_rng(5200 + it).standard_normal((mx, my)) * 1e-3
        Gd = to_dev(G)
        ec.eps_opt_step(p, opt, state, Cd, Gd, Md, Vd, ws, morph=morph)
        ec.eps_sync_status()
        C, M, V, s_new = oo.opt_step(oopt, s_ref, C, G.astype(np.float32).astype(np.float64), M, V, rho)
        st = ec.read_opt_state(state)
        slack = near_threshold(rho, oopt.gray_tol)
        assert st["step"] == it + 1
        assert st["gray_acc"] == 0 and st["ticket"] == 0
        assert abs(st["gray"] - s_new.gray) <= slack, (st["gray"], s_new.gray, slack)
        if st["gray"] == s_new.gray:
            for k in ("beta", "beta_max", "t", "unbinarity"):
                ref = getattr(s_new, k)
                assert abs(st[k] - ref) <= 2e-6 * abs(ref), (k, st[k], ref)
        np.testing.assert_allclose(Cd.cpu().numpy(), C, rtol=0, atol=2e-6)
        # M is a moving average of signed gradients and can cancel to near
        # zero: its FP32 error is bounded by a few ulp of the largest terms
        np.testing.assert_allclose(Md.cpu().numpy(), M, rtol=2e-5, atol=1e-6 * np.abs(M).max())
        np.testing.assert_allclose(Vd.cpu().numpy(), V, rtol=2e-5, atol=1e-16)
        s_ref = s_new
        results.append(st)
    return results


def test_one_step_matches_oracle():
    st = run_loop(1)
    assert st[0]["gray"] > 0


def test_four_iterations_match_oracle():
    st = run_loop(4)
    betas = [s["beta"] for s in st]
    assert betas == sorted(betas)


def test_real_cotangent_workspace():
    run_loop(2, real=True, mx=70, my=46)


def test_morphology_workspace():
    ec = _ec()
    run_loop(2, morph=ec.Morph(alpha=20.0, radius=2.0))


def test_binary_design_floors_unbinarity():
    # a binary design through the identity filter: every projected subpixel
    # is saturated, so gray = 0 and u is floored at one subpixel
    st = run_loop(1, binary=True, radius=1.0)
    assert st[0]["gray"] == 0
    assert st[0]["unbinarity"] == pytest.approx(1.0 / (64 * 64))
