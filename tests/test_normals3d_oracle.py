"""Pins of the 3-D face-normal oracle: the flat-design limit (n = z, the base
rule), the tensor invariant of a unit normal, a closed form for a linear
ramp, the mirror symmetry of the two faces, the 90-degree rotation, and
that nothing off the face planes changes."""

import numpy as np
import pytest

from oracle import epschain_oracle as orc
from oracle import normals3d_oracle as n3


def prob(mx=24, my=24, nz=16, radius=3.0, beta=8.0, bc=orc.CLAMP):
    return orc.Problem(mx=mx, my=my, nz=nz, radius=radius, beta=beta, bc=bc)


def test_flat_design_keeps_the_base_face_rule():
    p = prob(bc=orc.PERIODIC)
    C = np.full((24, 24), 0.57)
    eps, od = n3.forward_3d(p, C)
    base = orc.forward(p, C)["eps_hat"]
    np.testing.assert_allclose(eps, base, rtol=1e-14)
    assert np.abs(od).max() < 1e-14


def test_only_the_face_planes_change():
    rng = np.random.default_rng(1)
    p = prob(mx=20, my=28)
    C = rng.random((20, 28))
    eps, od = n3.forward_3d(p, C)
    fw = orc.forward(p, C, offdiag=True)
    faces = [p.k0, p.k0 + p.slab_nk]
    mask = np.ones(p.nz, bool)
    mask[faces] = False
    np.testing.assert_array_equal(eps[:2], fw["eps_hat"][:2])
    np.testing.assert_array_equal(eps[2][..., mask], fw["eps_hat"][2][..., mask])
    np.testing.assert_array_equal(od[:2], fw["offdiag"])
    assert np.all(od[2:][..., mask] == 0)
    assert np.abs(od[2:]).max() > 1e-3          # sidewalls meet the faces somewhere


def test_rows_of_a_unit_normal_tensor():
    # row z of T = (a - b) n n^T + b I with |n| = 1:
    # (T_zz - b)(a - b) = T_zx^2 + T_zy^2 + (T_zz - b)^2, and T_zz between b and a
    rng = np.random.default_rng(2)
    p = prob()
    C = rng.random((24, 24))
    eps, od = n3.forward_3d(p, C)
    fw = orc.forward(p, C)
    a = 0.5 * (fw["H"][2] + 1 / p.eps_clad)
    b = 1 / (0.5 * (fw["A"][2] + p.eps_clad))
    for k in (p.k0, p.k0 + p.slab_nk):
        t = 1 / eps[2, :, :, k] - b
        lhs = t * (a - b)
        rhs = od[2, :, :, k] ** 2 + od[3, :, :, k] ** 2 + t * t
        np.testing.assert_allclose(lhs, rhs, rtol=1e-10, atol=1e-16)
        lo, hi = np.minimum(a, b), np.maximum(a, b)
        assert np.all(1 / eps[2, :, :, k] >= lo - 1e-15) and np.all(1 / eps[2, :, :, k] <= hi + 1e-15)


def test_linear_ramp_closed_form():
    # C = alpha a + c0 (subpixel index a): the filter keeps it linear inside,
    # U_z rises by 2 alpha per Yee cell, the Sobel of U_z is 16 alpha, so
    # g = (8 alpha, 0, +-4 U_z) and n_x / n_z = +-2 alpha / U_z
    p = prob(mx=48, my=20, radius=2.0)
    alpha, c0 = 0.004, 0.3
    C = alpha * np.arange(48)[:, None] + c0 + 0 * np.arange(20)[None, :]
    eps, od = n3.forward_3d(p, C)
    fw = orc.forward(p, C)
    a = 0.5 * (fw["H"][2] + 1 / p.eps_clad)
    b = 1 / (0.5 * (fw["A"][2] + p.eps_clad))
    i = np.arange(4, 20)                           # cells away from the clamped edges
    Uz = orc.dual_cell_mean(fw["u"], 2, p)[i, 8]
    for k, s in ((p.k0, 1.0), (p.k0 + p.slab_nk, -1.0)):
        gx, gz = 8 * alpha, s * 4 * Uz
        g2 = gx * gx + gz * gz
        exp_zz = 1 / (gz * gz / g2 * a[i, 8] + (1 - gz * gz / g2) * b[i, 8])
        exp_zx = gz * gx / g2 * (a[i, 8] - b[i, 8])
        np.testing.assert_allclose(eps[2, i, 8, k], exp_zz, rtol=1e-12)
        np.testing.assert_allclose(od[2, i, 8, k], exp_zx, rtol=1e-10, atol=1e-16)
        np.testing.assert_allclose(od[3, i, 8, k], 0.0, atol=1e-15)


def test_faces_mirror_each_other():
    rng = np.random.default_rng(3)
    p = prob()
    eps, od = n3.forward_3d(p, rng.random((24, 24)))
    lo, hi = p.k0, p.k0 + p.slab_nk
    np.testing.assert_allclose(eps[2, :, :, lo], eps[2, :, :, hi], rtol=1e-14)
    np.testing.assert_allclose(od[2:, :, :, lo], -od[2:, :, :, hi], rtol=1e-14, atol=1e-18)


@pytest.mark.parametrize("bc", [orc.CLAMP, orc.PERIODIC])
def test_ninety_degree_rotation_swaps_x_and_y(bc):
    rng = np.random.default_rng(4)
    p = prob(bc=bc)
    C = rng.random((24, 24))
    eps, od = n3.forward_3d(p, C)
    eps_t, od_t = n3.forward_3d(p, C.T.copy())
    k = p.k0
    np.testing.assert_allclose(eps_t[2, :, :, k], eps[2, :, :, k].T, rtol=1e-13)
    np.testing.assert_allclose(od_t[2, :, :, k], od[3, :, :, k].T, rtol=1e-12, atol=1e-16)
    np.testing.assert_allclose(od_t[3, :, :, k], od[2, :, :, k].T, rtol=1e-12, atol=1e-16)
