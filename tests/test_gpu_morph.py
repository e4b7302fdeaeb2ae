"""Chain with morphological filtering (Eq. 3-6): the CUDA path (through the
C ABI) against the FP64 morphology oracle, element by element.

Tolerances as for the base chain (FP32 path, beta <= 32):
  eps_hat:  max |gpu - ref| / |ref|            <= 1e-5
  dJ/dC:    max |gpu - ref| / max |ref|        <= 1e-4
"""

import numpy as np
import pytest

from oracle import epschain_oracle as orc
from oracle import morph_oracle as mo
from paper_2505_03352_gb300 import synth

pytestmark = pytest.mark.gpu

EPS_TOL = 1e-5
GRAD_TOL = 1e-4
D, E = mo.DILATE, mo.ERODE


def _ec():
    import paper_2505_03352_gb300 as ec
    return ec


def to_dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def eps_err(got, ref):
    return float(np.max(np.abs(got - ref) / np.abs(ref)))


def grad_err(got, ref):
    return float(np.max(np.abs(got - ref)) / np.max(np.abs(ref)))


def case(mx, my, nz, radius, beta, bc, mr, alpha, ops, seed):
    ec = _ec()
    p = ec.Problem(mx=mx, my=my, nz=nz, radius=radius, beta=beta, bc=bc)
    o = orc.Problem(mx=mx, my=my, nz=nz, radius=radius, beta=beta, bc=bc)
    m = ec.Morph(alpha=alpha, radius=mr, ops=tuple(ops))
    om = mo.Morph(alpha=alpha, radius=mr, ops=tuple(ops))
    C = synth.soi_layout(mx, my, seed, sigma=3.0)
    shape = (3, p.nx, p.ny, p.nz)
    EF = [synth.complex_field(shape, seed + 1)]
    EA = [synth.complex_field(shape, seed + 2)]
    return p, o, m, om, C, EF, EA


def check(p, o, m, om, C, EF, EA):
    ec = _ec()
    ref = mo.eps_hat_morph(o, om, C)
    e = ec.eps_forward_morph(p, m, to_dev(C)).cpu().numpy()
    ec.eps_sync_status()
    assert eps_err(e, ref) <= EPS_TOL, ("eps", eps_err(e, ref))
    ref_g = mo.vjp_fields_morph(o, om, C, EF, EA)
    g, e2 = ec.eps_vjp_morph(p, m, to_dev(C), [to_dev(x) for x in EF], [to_dev(x) for x in EA],
                             eps_out=True)
    ec.eps_sync_status()
    g, e2 = g.cpu().numpy(), e2.cpu().numpy()
    assert np.abs(ref_g).max() > 0
    assert grad_err(g, ref_g) <= GRAD_TOL, ("grad", grad_err(g, ref_g))
    assert eps_err(e2, ref) <= EPS_TOL
    # real cotangent
    G = np.random.default_rng(5).standard_normal((3, p.nx, p.ny, p.nz)).astype(np.float32)
    ref_r = mo.vjp_real_morph(o, om, C, G.astype(np.float64))
    gr = ec.eps_vjp_real_morph(p, m, to_dev(C), to_dev(G)).cpu().numpy()
    ec.eps_sync_status()
    assert grad_err(gr, ref_r) <= GRAD_TOL, ("real", grad_err(gr, ref_r))
    return grad_err(g, ref_g)


CLOSE_OPEN = (D, E, E, D)


@pytest.mark.parametrize("mx,my,nz,radius,beta,bc,mr,alpha,ops", [
    (64, 64, 16, 3.0, 8.0, 0, 2.0, 20.0, CLOSE_OPEN),       # cfg1 shape, App. B alpha
    (64, 64, 16, 3.0, 8.0, 1, 2.0, 20.0, CLOSE_OPEN),       # periodic
    (70, 46, 16, 2.5, 16.0, 0, 1.5, 20.0, (D,)),            # ragged tiles, one dilate
    (38, 102, 14, 4.0, 16.0, 1, 3.5, 30.0, (E, D)),          # ragged, opening, periodic
    (96, 66, 16, 3.0, 32.0, 0, 1.0, 20.0, CLOSE_OPEN),       # beta = 32
    (8, 10, 14, 2.0, 8.0, 0, 4.0, 20.0, CLOSE_OPEN),         # domain smaller than the disk halo
    (8, 10, 14, 2.0, 8.0, 1, 4.0, 20.0, (D, E)),             # same, wrapped
    (64, 64, 16, 3.0, 8.0, 0, 2.0, 20.0, ()),                # no operations: two projections
    (64, 64, 16, 3.0, 8.0, 0, 0.0, 20.0, (D, E)),            # one-point disk: identity operations
    (34, 34, 16, 1.0, 8.0, 0, 2.0, 20.0, CLOSE_OPEN),        # identity conic filter
    (128, 96, 16, 6.0, 16.0, 0, 7.5, 20.0, CLOSE_OPEN),      # d = 150 nm at 10 nm pitch
    (66, 70, 16, 3.0, 8.0, 0, 11.5, 60.0, (E, D, D, E, D, E, E, D)),   # largest disk, alpha, ops
])
def test_morph_chain_matches_oracle(mx, my, nz, radius, beta, bc, mr, alpha, ops):
    check(*case(mx, my, nz, radius, beta, bc, mr, alpha, ops, seed=4100 + mx + my))


def test_morph_chain_cfg2_size():
    # cfg2 controls (600 x 600, R = 6, beta = 16, nz = 24) with the App. B
    # morphology (alpha = 20) and a 20 nm-radius disk, closing then opening
    w = synth.WORKLOADS[2]
    ec = _ec()
    p = ec.Problem(mx=w.mx, my=w.my, nz=w.nz, radius=w.radius, beta=w.beta)
    o = orc.Problem(mx=w.mx, my=w.my, nz=w.nz, radius=w.radius, beta=w.beta)
    m, om = ec.Morph(alpha=20.0, radius=2.0), mo.Morph(alpha=20.0, radius=2.0)
    C = synth.controls(w)
    EF, EA = synth.fields(w)
    check(p, o, m, om, C, EF, EA)


def test_morph_autograd_matches_oracle():
    import torch
    from paper_2505_03352_gb300.autograd import eps_chain_morph
    p, o, m, om, C, _, _ = case(48, 40, 16, 3.0, 8.0, 0, 2.0, 20.0, CLOSE_OPEN, seed=4300)
    Ct = to_dev(C).requires_grad_(True)
    eps = eps_chain_morph(Ct, p, m)
    G = np.random.default_rng(6).standard_normal(tuple(eps.shape)).astype(np.float32)
    (eps * to_dev(G)).sum().backward()
    ref = mo.vjp_real_morph(o, om, C, G.astype(np.float64))
    assert grad_err(Ct.grad.cpu().numpy(), ref) <= GRAD_TOL
    assert eps_err(eps.detach().cpu().numpy(), mo.eps_hat_morph(o, om, C)) <= EPS_TOL
    torch.cuda.synchronize()


def test_morph_repeated_calls_are_bitwise_identical():
    ec = _ec()
    p, _, m, _, C, EF, EA = case(96, 64, 16, 3.0, 16.0, 0, 2.5, 20.0, CLOSE_OPEN, seed=4400)
    Cd, EFd, EAd = to_dev(C), [to_dev(x) for x in EF], [to_dev(x) for x in EA]
    a = ec.eps_vjp_morph(p, m, Cd, EFd, EAd).cpu().numpy()
    b = ec.eps_vjp_morph(p, m, Cd, EFd, EAd).cpu().numpy()
    ec.eps_sync_status()
    assert np.array_equal(a, b)
