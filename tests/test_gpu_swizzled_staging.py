"""eps_hat through the stencil's swizzled staging (nz = 32: each column's
planes are one 128-byte swizzle row, one 4-D tensor store per component).

The forms that use it (eps_forward at nz = 32; the fused call's eps_out at
nz = 32, within one wave of tiles with three staging buffers and beyond it
with one) are checked against the FP64 oracle within the forward's
tolerance (eps_hat 1e-5 relative), on shapes whose last tile row and column
are partial, so the tensor store's clipping at the region edge is
exercised.  The forms agree with each other bit for bit, and with the plain
staging of the batched launch (which never takes the swizzled form)."""

import numpy as np
import pytest

from oracle import epschain_oracle as orc
from oracle import normals3d_oracle as n3
from paper_2505_03352_gb300 import synth

pytestmark = pytest.mark.gpu

EPS_TOL = 1e-5


def _dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _eps_err(got, ref):
    return float(np.max(np.abs(got - ref) / np.abs(ref)))


# (mx, my): one wave of tiles (60 x 100 columns: 8 x 4 tiles, both partial),
# several waves (601 x 521 columns: 76 x 17 tiles, both partial), and a
# single partial tile (3 x 5 columns)
@pytest.mark.parametrize("mx,my,bc", [(120, 200, 0), (1202, 1042, 1), (6, 10, 0)])
def test_swizzled_forward_matches_the_oracle(mx, my, bc):
    import paper_2505_03352_gb300 as ec
    nz = 32
    p = ec.Problem(mx=mx, my=my, nz=nz, radius=6.0, beta=16.0, bc=bc)
    o = orc.Problem(mx=mx, my=my, nz=nz, radius=6.0, beta=16.0, bc=bc)
    C = synth.soi_layout(mx, my, 8700 + mx)
    eps = ec.eps_forward(p, _dev(C))
    ec.eps_sync_status()
    assert _eps_err(eps.cpu().numpy(), orc.eps_hat(o, C)) <= EPS_TOL


@pytest.mark.parametrize("mx,my", [(120, 200), (1202, 1042)])
def test_fused_eps_out_swizzled_equals_forward_and_batched(mx, my):
    import paper_2505_03352_gb300 as ec
    nz = 32
    p = ec.Problem(mx=mx, my=my, nz=nz, radius=6.0, beta=16.0)
    C = _dev(synth.soi_layout(mx, my, 8800 + mx))
    eps = ec.eps_forward(p, C)
    zero = [_dev(np.zeros((3, p.nx, p.ny, nz), np.complex64))]
    _, fused = ec.eps_vjp(p, C, zero, zero, eps_out=True)
    batched = ec.eps_forward_batched([p], [C])[0]
    ec.eps_sync_status()
    e = eps.cpu().numpy()
    np.testing.assert_array_equal(e, fused.cpu().numpy())
    np.testing.assert_array_equal(e, batched.cpu().numpy())


def test_swizzled_forward_with_3d_normals_matches_the_oracle():
    # 3-D face normals change eps_zz on the face planes only; without the
    # off-diagonal maps the eps_hat components take the swizzled form
    import paper_2505_03352_gb300 as ec
    mx, my, nz = 402, 330, 32
    p = ec.Problem(mx=mx, my=my, nz=nz, radius=3.0, beta=8.0, flags=ec.EPS_FLAG_NORMALS_3D)
    o = orc.Problem(mx=mx, my=my, nz=nz, radius=3.0, beta=8.0)
    C = synth.soi_layout(mx, my, 8900, sigma=3.0)
    eps = ec.eps_forward(p, _dev(C))
    ec.eps_sync_status()
    ref_e, _ = n3.forward_3d(o, C)
    assert _eps_err(eps.cpu().numpy(), ref_e) <= EPS_TOL
