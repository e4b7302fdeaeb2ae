"""3-D normals at the slab faces and the Ez row of the inverse-permittivity
tensor (EPS_FLAG_NORMALS_3D): the CUDA forward against the FP64 oracle.
eps_hat: max relative error <= 1e-5; off-diagonal maps (they cross zero):
max |delta| / max |ref| <= 1e-4, as for the base chain's xy term."""

import numpy as np
import pytest

from oracle import epschain_oracle as orc
from oracle import normals3d_oracle as n3
from paper_2505_03352_gb300 import synth

pytestmark = pytest.mark.gpu


def _ec():
    import paper_2505_03352_gb300 as ec
    return ec


def to_dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


@pytest.mark.parametrize("mx,my,nz,radius,beta,bc,with_od", [
    (70, 98, 16, 3.0, 8.0, 0, True),
    (70, 98, 16, 3.0, 8.0, 1, True),
    (64, 64, 24, 6.0, 32.0, 0, True),
    (46, 30, 15, 2.5, 16.0, 0, True),        # nz not a multiple of 4: direct stores
    (600, 600, 24, 6.0, 16.0, 0, True),      # cfg2 size
    (64, 64, 16, 3.0, 8.0, 0, False),        # eps_hat only
])
def test_normals3d_forward_matches_oracle(mx, my, nz, radius, beta, bc, with_od):
    ec = _ec()
    flags = ec.EPS_FLAG_NORMALS_3D | (ec.EPS_FLAG_OFFDIAG if with_od else 0)
    p = ec.Problem(mx=mx, my=my, nz=nz, radius=radius, beta=beta, bc=bc, flags=flags)
    o = orc.Problem(mx=mx, my=my, nz=nz, radius=radius, beta=beta, bc=bc)
    C = synth.soi_layout(mx, my, 7000 + mx, sigma=3.0)
    out = ec.eps_forward(p, to_dev(C))
    ec.eps_sync_status()
    eps, od = (out[0].cpu().numpy(), out[1].cpu().numpy()) if with_od else (out.cpu().numpy(), None)
    ref_e, ref_od = n3.forward_3d(o, C)
    assert float(np.max(np.abs(eps - ref_e) / ref_e)) <= 1e-5
    if with_od:
        assert od.shape == (4, p.nx, p.ny, nz)
        err = float(np.max(np.abs(od - ref_od)) / np.max(np.abs(ref_od)))
        assert err <= 1e-4, err
        assert np.abs(ref_od[2:]).max() > 1e-3


def test_normals3d_is_forward_only():
    ec = _ec()
    p = ec.Problem(mx=32, my=32, nz=16, radius=3.0, beta=8.0, flags=ec.EPS_FLAG_NORMALS_3D)
    C = to_dev(np.full((32, 32), 0.5, np.float32))
    G = to_dev(np.zeros((3, 16, 16, 16), np.float32))
    with pytest.raises(ec.EpsError):
        ec.eps_vjp_real(p, C, G)
