"""Pins of the morphology oracle (Eq. 3-6) to what the mathematics fixes:
the hard max / min limit of the soft operations (against scipy's grey
morphology), fixed points, a brute-force disk sum, duality, the
closing/opening behaviour on binary features, and complex-step and
finite-difference derivatives of the whole chain."""

import numpy as np
import pytest
from scipy import ndimage

from oracle import epschain_oracle as orc
from oracle import morph_oracle as mo

CLAMP, PERIODIC = orc.CLAMP, orc.PERIODIC
SCIPY_MODE = {CLAMP: "nearest", PERIODIC: "wrap"}


def footprint(radius):
    n = int(np.floor(radius))
    p, q = np.mgrid[-n:n + 1, -n:n + 1]
    return p * p + q * q <= radius * radius


@pytest.mark.parametrize("radius,count", [(0.0, 1), (1.0, 5), (1.5, 9), (2.0, 13), (2.5, 21), (3.0, 29)])
def test_disk_taps_are_the_lattice_points_of_the_closed_disk(radius, count):
    taps = mo.disk_taps(radius)
    assert len(taps) == count                      # Gauss circle counts
    assert abs(sum(w for _, _, w in taps) - 1.0) < 1e-15


@pytest.mark.parametrize("bc", [CLAMP, PERIODIC])
def test_disk_sum_matches_a_loop_over_neighbours(bc):
    rng = np.random.default_rng(1)
    f = rng.random((6, 7))
    got = mo.disk_sum(f, 1.5, bc)
    for x in range(6):
        for y in range(7):
            vals = []
            for p in range(-1, 2):
                for q in range(-1, 2):
                    a, b = x + p, y + q
                    if bc == CLAMP:
                        a, b = min(max(a, 0), 5), min(max(b, 0), 6)
                    else:
                        a, b = a % 6, b % 7
                    vals.append(f[a, b])
            assert abs(got[x, y] - np.mean(vals)) < 1e-14


@pytest.mark.parametrize("bc", [CLAMP, PERIODIC])
@pytest.mark.parametrize("radius", [1.0, 2.5, 4.0])
def test_uniform_density_is_a_fixed_point(bc, radius):
    m = mo.Morph(alpha=20.0, radius=radius)
    rho = np.full((12, 10), 0.37)
    np.testing.assert_allclose(mo.dilate(rho, m, bc), rho, rtol=0, atol=1e-14)
    np.testing.assert_allclose(mo.erode(rho, m, bc), rho, rtol=0, atol=1e-14)


def test_radius_zero_is_the_identity():
    rng = np.random.default_rng(2)
    rho = rng.random((9, 9))
    m = mo.Morph(alpha=20.0, radius=0.0)
    np.testing.assert_allclose(mo.dilate(rho, m, CLAMP), rho, rtol=0, atol=1e-14)
    np.testing.assert_allclose(mo.erode(rho, m, CLAMP), rho, rtol=0, atol=1e-14)


@pytest.mark.parametrize("bc", [CLAMP, PERIODIC])
@pytest.mark.parametrize("radius", [1.0, 2.0, 3.5])
def test_large_alpha_tends_to_grey_max_and_min(bc, radius):
    # normalised disk of N points:  max - log(N)/alpha <= dilate <= max,
    # min <= erode <= min + log(N)/alpha
    rng = np.random.default_rng(3)
    rho = rng.random((20, 17))
    alpha = 500.0
    m = mo.Morph(alpha=alpha, radius=radius)
    fp = footprint(radius)
    slack = np.log(fp.sum()) / alpha
    dmax = ndimage.grey_dilation(rho, footprint=fp, mode=SCIPY_MODE[bc])
    emin = ndimage.grey_erosion(rho, footprint=fp, mode=SCIPY_MODE[bc])
    d = mo.dilate(rho, m, bc)
    e = mo.erode(rho, m, bc)
    assert np.all(d <= dmax + 1e-12) and np.all(d >= dmax - slack - 1e-12)
    assert np.all(e >= emin - 1e-12) and np.all(e <= emin + slack + 1e-12)


@pytest.mark.parametrize("bc", [CLAMP, PERIODIC])
def test_soft_operations_bracket_the_disk_mean(bc):
    # log-mean-exp >= mean (Jensen): dilate >= disk mean >= erode
    rng = np.random.default_rng(4)
    rho = rng.random((15, 15))
    m = mo.Morph(alpha=20.0, radius=2.0)
    mean = mo.disk_sum(rho, 2.0, bc)
    assert np.all(mo.dilate(rho, m, bc) >= mean - 1e-14)
    assert np.all(mo.erode(rho, m, bc) <= mean + 1e-14)


def test_erode_is_dual_to_dilate():
    rng = np.random.default_rng(5)
    rho = rng.random((11, 13))
    m = mo.Morph(alpha=20.0, radius=2.0)
    np.testing.assert_allclose(mo.erode(rho, m, CLAMP), 1.0 - mo.dilate(1.0 - rho, m, CLAMP),
                               rtol=0, atol=1e-14)


def test_closing_fills_a_hole_and_opening_removes_an_island():
    rho = np.zeros((24, 24))
    rho[2:12, 2:12] = 1.0          # solid square with a one-pixel hole
    rho[6, 6] = 0.0
    rho[18, 18] = 1.0              # one-pixel island in the void
    m = mo.Morph(alpha=400.0, radius=1.0)
    slack = 2 * np.log(5) / 400.0
    closed = mo.erode(mo.dilate(rho, m, CLAMP), m, CLAMP)
    opened = mo.dilate(mo.erode(rho, m, CLAMP), m, CLAMP)
    assert closed[6, 6] > 1.0 - slack
    assert opened[18, 18] < slack
    # against scipy's hard closing / opening with the same disk
    fp = footprint(1.0)
    np.testing.assert_allclose(closed, ndimage.grey_closing(rho, footprint=fp, mode="nearest"),
                               atol=slack)
    np.testing.assert_allclose(opened, ndimage.grey_opening(rho, footprint=fp, mode="nearest"),
                               atol=slack)


@pytest.mark.parametrize("op", [mo.DILATE, mo.ERODE])
@pytest.mark.parametrize("bc", [CLAMP, PERIODIC])
def test_single_operation_transpose_matches_complex_step(op, bc):
    rng = np.random.default_rng(6)
    rho = rng.random((7, 6))
    m = mo.Morph(alpha=20.0, radius=1.5, ops=(op,))
    f = mo.dilate if op == mo.DILATE else mo.erode
    h = 1e-30
    J = np.zeros((rho.size, rho.size))
    for i in range(rho.size):
        z = rho.astype(np.complex128)
        z.flat[i] += 1j * h
        J[:, i] = np.imag(f(z, m, bc)).ravel() / h
    assert np.all(J >= -1e-15)                       # softmax weights are positive
    g = rng.standard_normal(rho.shape)
    np.testing.assert_allclose(mo.morph_op_T(rho, g, op, m, bc), (J.T @ g.ravel()).reshape(rho.shape),
                               rtol=1e-12, atol=1e-12)


def _prob(bc=CLAMP, mx=8, my=8, nz=14, radius=2.0, beta=8.0):
    return orc.Problem(mx=mx, my=my, nz=nz, radius=radius, beta=beta, bc=bc)


@pytest.mark.parametrize("bc", [CLAMP, PERIODIC])
def test_chain_vjp_matches_complex_step_jacobian(bc):
    rng = np.random.default_rng(7)
    p = _prob(bc=bc)
    m = mo.Morph(alpha=20.0, radius=1.5)
    C = 0.5 + 0.3 * rng.standard_normal((8, 8))
    h = 1e-30
    J = np.zeros((3 * p.nx * p.ny * p.nz, C.size))
    for i in range(C.size):
        z = C.astype(np.complex128)
        z.flat[i] += 1j * h
        J[:, i] = np.imag(mo.eps_hat_morph(p, m, z)).ravel() / h
    assert np.abs(J).max() > 0.1
    G = rng.standard_normal((3, p.nx, p.ny, p.nz))
    ref = (J.T @ G.ravel()).reshape(C.shape)
    np.testing.assert_allclose(mo.vjp_real_morph(p, m, C, G), ref, rtol=1e-10,
                               atol=1e-10 * np.abs(ref).max())


def test_chain_vjp_central_finite_differences():
    rng = np.random.default_rng(8)
    p = _prob(mx=24, my=20, nz=16, radius=3.0, beta=8.0)
    m = mo.Morph(alpha=20.0, radius=2.0)
    C = np.clip(rng.random((24, 20)) * 1.2 - 0.1, 0, 1)
    shape = (3, p.nx, p.ny, p.nz)
    EF = [rng.standard_normal(shape) + 1j * rng.standard_normal(shape)]
    EA = [rng.standard_normal(shape) + 1j * rng.standard_normal(shape)]
    G = orc.field_cotangent(p, EF, EA)
    grad = mo.vjp_fields_morph(p, m, C, EF, EA)
    np.testing.assert_allclose(grad, mo.vjp_real_morph(p, m, C, G), rtol=0, atol=1e-13)
    hstep = 1e-6
    for idx in rng.choice(C.size, 10, replace=False):
        Cp, Cm = C.copy(), C.copy()
        Cp.flat[idx] += hstep
        Cm.flat[idx] -= hstep
        fd = (np.sum(G * mo.eps_hat_morph(p, m, Cp)) - np.sum(G * mo.eps_hat_morph(p, m, Cm))) / (2 * hstep)
        assert abs(fd - grad.flat[idx]) <= 1e-6 * max(1.0, np.abs(grad).max())


def test_uniform_controls_give_the_uniform_closed_form():
    # uniform C -> uniform u = c, rho0 = P(c), morphology keeps it, and the
    # Yee stage sees a uniform density: every slab voxel is eps_sub(P(rho0 - 1/2))
    p = _prob(mx=12, my=12, nz=16, radius=3.0, beta=8.0, bc=PERIODIC)
    m = mo.Morph(alpha=20.0, radius=2.0)
    c = 0.58
    rho0 = 0.5 * (1 + np.tanh(8.0 * (c - 0.5)))
    rho = 0.5 * (1 + np.tanh(8.0 * (rho0 - 0.5)))
    e = p.eps_clad + rho * (p.eps_core - p.eps_clad)
    eh = mo.eps_hat_morph(p, m, np.full((12, 12), c))
    lo, hi = orc.support_planes(p)["xy"]
    np.testing.assert_allclose(eh[0, :, :, lo:hi], e, rtol=1e-13)
    np.testing.assert_allclose(eh[1, :, :, lo:hi], e, rtol=1e-13)
    np.testing.assert_allclose(eh[2, :, :, lo:hi - 1], e, rtol=1e-13)
