"""eps_forward beyond one wave of tiles at nz other than 32 (nz = 32 takes
the swizzled staging instead), where eps_hat leaves by warp-cooperative
direct stores instead of shared-memory staging: the same
values as the staged write of the fused call (bit for bit), and, with the
off-diagonal maps and 3-D face normals, the FP64 oracle within the
forward's tolerances (eps_hat 1e-5 relative; off-diagonal maps 1e-4 of
their largest value)."""

import numpy as np
import pytest

from oracle import epschain_oracle as orc
from oracle import normals3d_oracle as n3
from paper_2505_03352_gb300 import synth

pytestmark = pytest.mark.gpu


def _dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


# 1600 x 1200 (800 x 600 columns, 1900 tiles) and a ragged 1202 x 1042 (601
# x 521 columns: a partial last tile row and column), both rules
@pytest.mark.parametrize("mx,my,nz,bc", [(1600, 1200, 28, 0), (1202, 1042, 24, 1)])
def test_direct_stores_equal_the_staged_write(mx, my, nz, bc):
    import paper_2505_03352_gb300 as ec
    p = ec.Problem(mx=mx, my=my, nz=nz, radius=6.0, beta=16.0, bc=bc)
    C = _dev(synth.soi_layout(mx, my, 8100 + mx))
    eps = ec.eps_forward(p, C)
    zero = [_dev(np.zeros((3, p.nx, p.ny, nz), np.complex64))]
    _, staged = ec.eps_vjp(p, C, zero, zero, eps_out=True)
    ec.eps_sync_status()
    np.testing.assert_array_equal(eps.cpu().numpy(), staged.cpu().numpy())


def test_direct_stores_with_offdiagonal_and_3d_normals_match_the_oracle():
    import paper_2505_03352_gb300 as ec
    mx = my = 1000                     # 500 x 500 columns: 1008 tiles
    nz = 16
    flags = ec.EPS_FLAG_NORMALS_3D | ec.EPS_FLAG_OFFDIAG
    p = ec.Problem(mx=mx, my=my, nz=nz, radius=3.0, beta=8.0, flags=flags)
    o = orc.Problem(mx=mx, my=my, nz=nz, radius=3.0, beta=8.0)
    C = synth.soi_layout(mx, my, 8300, sigma=3.0)
    eps, od = ec.eps_forward(p, _dev(C))
    ec.eps_sync_status()
    ref_e, ref_od = n3.forward_3d(o, C)
    assert float(np.max(np.abs(eps.cpu().numpy() - ref_e) / ref_e)) <= 1e-5
    err = float(np.max(np.abs(od.cpu().numpy() - ref_od)) / np.max(np.abs(ref_od)))
    assert err <= 1e-4, err
