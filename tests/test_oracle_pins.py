"""Pins of the FP64 oracle to what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: closed
forms, invariants, limits stated in the paper, a geometric brute force of
the dual cells, complex-step derivatives and central finite differences.
"""

import numpy as np
import pytest

from oracle import epschain_oracle as orc
from tests import _geometry_bruteforce as bf

CLAMP, PERIODIC = orc.CLAMP, orc.PERIODIC


def prob(mx=16, my=16, nz=16, radius=3.0, beta=8.0, bc=CLAMP, **kw):
    return orc.Problem(mx=mx, my=my, nz=nz, radius=radius, beta=beta, bc=bc, **kw)


# ---------------------------------------------------------------- filter (Eq. 2)

@pytest.mark.parametrize("bc", [CLAMP, PERIODIC])
@pytest.mark.parametrize("radius", [1.0, 2.5, 3.0, 6.0])
def test_filter_uniform_stays_uniform(bc, radius):
    C = np.full((20, 14), 0.37)
    u = orc.filter_density(C, radius, bc)
    np.testing.assert_allclose(u, 0.37, rtol=0, atol=1e-15)


@pytest.mark.parametrize("radius", [2.0, 3.0, 4.5, 6.0, 8.0])
def test_filter_periodic_preserves_mean(radius):
    rng = np.random.default_rng(0)
    C = rng.random((24, 18))
    u = orc.filter_density(C, radius, PERIODIC)
    assert abs(u.sum() - C.sum()) < 1e-12 * C.size


@pytest.mark.parametrize("bc", [CLAMP, PERIODIC])
@pytest.mark.parametrize("radius", [0.3, 1.0])
def test_filter_small_radius_is_identity(bc, radius):
    rng = np.random.default_rng(1)
    C = rng.random((10, 12))
    np.testing.assert_array_equal(orc.filter_density(C, radius, bc), C)


@pytest.mark.parametrize("radius,count", [(3.0, 25), (6.0, 109), (8.0, 193)])
def test_filter_delta_response_is_a_cone(radius, count):
    n = 41
    c = n // 2
    C = np.zeros((n, n))
    C[c, c] = 1.0
    u = orc.filter_density(C, radius, PERIODIC)
    # support: the open disk r < R (lattice-point count of the disk)
    assert np.count_nonzero(u) == count
    assert abs(u.sum() - 1.0) < 1e-14
    # 8-fold symmetry of the square lattice
    np.testing.assert_allclose(u, u.T, atol=1e-17)
    np.testing.assert_allclose(u, u[::-1, :], atol=1e-17)
    np.testing.assert_allclose(u, u[:, ::-1], atol=1e-17)
    # along an axis the profile falls linearly and would reach 0 at r = R
    p = np.arange(int(np.ceil(radius)))
    prof = u[c, c + p] / u[c, c]
    np.testing.assert_allclose(prof, 1.0 - p / radius, atol=1e-14)
    # on the diagonal the same cone: value depends on r only
    d = 2
    np.testing.assert_allclose(u[c + d, c + d] / u[c, c], 1.0 - np.hypot(d, d) / radius,
                               atol=1e-14)


def test_filter_transpose_is_adjoint():
    rng = np.random.default_rng(2)
    for bc in (CLAMP, PERIODIC):
        C = rng.random((13, 11))
        du = rng.standard_normal((13, 11))
        lhs = np.sum(orc.filter_density(C, 3.5, bc) * du)
        rhs = np.sum(C * orc.filter_density_T(du, 3.5, bc))
        assert abs(lhs - rhs) < 1e-12


def test_filter_clamp_edge_replicates():
    # a step that touches the lower-x edge: replicate means the edge rows
    # see C as if the region continued with its edge value.
    C = np.zeros((12, 12))
    C[:3, :] = 1.0
    u = orc.filter_density(C, 2.0, CLAMP)
    np.testing.assert_allclose(u[0, :], 1.0, atol=1e-15)


# ------------------------------------------------------- projection (Eq. 3/6)

def test_projection_limits_and_symmetry():
    u = np.linspace(-0.5, 1.5, 401)
    for beta in (4.0, 8.0, 32.0):
        rho = orc.project(u, beta, 0.5)
        assert np.all((rho >= 0) & (rho <= 1))
        np.testing.assert_allclose(rho + orc.project(1.0 - u, beta, 0.5), 1.0, atol=1e-15)
    assert orc.project(np.array([0.5]), 16.0, 0.5)[0] == 0.5
    # beta -> infinity gives a binary design (Sec. 3)
    rho = orc.project(u[np.abs(u - 0.5) > 1e-3], 1e6, 0.5)
    assert set(np.unique(rho)) <= {0.0, 1.0}


def test_projection_derivative_matches_central_difference():
    u = np.linspace(0.2, 0.8, 37)
    for beta in (4.0, 32.0):
        h = 1e-7
        fd = (orc.project(u + h, beta, 0.45) - orc.project(u - h, beta, 0.45)) / (2 * h)
        np.testing.assert_allclose(orc.project_grad(u, beta, 0.45), fd, rtol=1e-6, atol=1e-9)


def test_mixing_endpoints():
    assert orc.mix(np.array(0.0), 12.11, 2.085) == 2.085
    assert orc.mix(np.array(1.0), 12.11, 2.085) == 12.11


# ------------------------------------------------- dual-cell means (Eq. 8)

@pytest.mark.parametrize("bc", [CLAMP, PERIODIC])
@pytest.mark.parametrize("shape", [(8, 8), (12, 10)])
def test_dual_cell_means_match_geometric_bruteforce(bc, shape):
    rng = np.random.default_rng(3)
    f = rng.random(shape)
    p = prob(mx=shape[0], my=shape[1], bc=bc)
    for c in range(3):
        got = orc.dual_cell_mean(f, c, p)
        ref = bf.all_box_averages(f, c, p.nx, p.ny, p.sub, bc)
        np.testing.assert_allclose(got, ref, rtol=0, atol=1e-15)


def test_dual_cell_mean_transpose_is_adjoint():
    rng = np.random.default_rng(4)
    for bc in (CLAMP, PERIODIC):
        p = prob(mx=10, my=12, bc=bc)
        f = rng.random((10, 12))
        for c in range(3):
            g = rng.standard_normal((p.nx, p.ny))
            lhs = np.sum(orc.dual_cell_mean(f, c, p) * g)
            rhs = np.sum(f * orc.dual_cell_mean_T(g, c, p))
            assert abs(lhs - rhs) < 1e-12


# -------------------------------------------------------- normals (Sec. 3)

@pytest.mark.parametrize("alpha,gamma", [(1.0, 0.0), (0.0, 1.0), (1.0, 1.0), (0.3, -0.7), (-2.0, 0.5)])
def test_sobel_normals_of_a_linear_ramp(alpha, gamma):
    # R < 1 makes u = C, so the averaged density is linear in (i, j) and the
    # Sobel gradient is exact there: m_x = alpha^2 / (alpha^2 + gamma^2).
    n = 20
    a = np.arange(n)[:, None]
    b = np.arange(n)[None, :]
    C = 0.5 + 0.01 * (alpha * a + gamma * b)
    p = prob(mx=n, my=n, radius=0.5, bc=CLAMP)
    fw = orc.forward(p, C)
    inner = (slice(2, p.nx - 2), slice(2, p.ny - 2))
    mx_ref = alpha ** 2 / (alpha ** 2 + gamma ** 2)
    np.testing.assert_allclose(fw["m"][0][inner], mx_ref, atol=1e-12)
    np.testing.assert_allclose(fw["m"][1][inner], 1.0 - mx_ref, atol=1e-12)


def test_sobel_transpose_is_adjoint():
    rng = np.random.default_rng(5)
    for bc in (CLAMP, PERIODIC):
        U = rng.random((7, 9))
        dgx, dgy = rng.standard_normal((2, 7, 9))
        gx, gy = orc.sobel(U, bc)
        lhs = np.sum(gx * dgx + gy * dgy)
        rhs = np.sum(U * orc.sobel_T(dgx, dgy, bc))
        assert abs(lhs - rhs) < 1e-12


# --------------------------------------------- Eq. 7, z rules, closed forms

@pytest.mark.parametrize("bc", [CLAMP, PERIODIC])
@pytest.mark.parametrize("c", [0.0, 0.2, 0.5, 0.83, 1.0])
def test_uniform_design_closed_form(bc, c):
    p = prob(mx=16, my=12, nz=16, radius=3.0, beta=8.0, bc=bc)
    C = np.full((16, 12), c)
    eh = orc.eps_hat(p, C)
    rho = 0.5 * (1 + np.tanh(8.0 * (c - 0.5)))
    es = 2.085 + rho * (12.11 - 2.085)
    k0, nk = p.k0, p.slab_nk
    assert k0 == 2
    np.testing.assert_allclose(eh[0, :, :, k0 + 1:k0 + nk + 1], es, rtol=1e-14)
    np.testing.assert_allclose(eh[1, :, :, k0 + 1:k0 + nk + 1], es, rtol=1e-14)
    np.testing.assert_allclose(eh[2, :, :, k0 + 1:k0 + nk], es, rtol=1e-14)
    face = 1.0 / (0.5 / es + 0.5 / 2.085)      # harmonic mean of slab and cladding
    np.testing.assert_allclose(eh[2, :, :, k0], face, rtol=1e-14)
    np.testing.assert_allclose(eh[2, :, :, k0 + nk], face, rtol=1e-14)
    clad = np.ones(16, bool)
    clad[k0 + 1:k0 + nk + 1] = False
    np.testing.assert_array_equal(eh[0][..., clad], 2.085)
    np.testing.assert_array_equal(eh[1][..., clad], 2.085)
    zclad = np.ones(16, bool)
    zclad[k0:k0 + nk + 1] = False
    np.testing.assert_array_equal(eh[2][..., zclad], 2.085)


def test_uniform_half_density_is_average_permittivity():
    # Sec. 4: a uniform block at the projection midpoint has the average of
    # core and cladding permittivity.
    p = prob(mx=8, my=8, beta=32.0)
    eh = orc.eps_hat(p, np.full((8, 8), 0.5))
    np.testing.assert_allclose(eh[0, :, :, p.k0 + 1], 0.5 * (12.11 + 2.085), rtol=1e-13)


def _box_means(e, comp, p):
    """Arithmetic and harmonic mean of e over each box, from the brute force."""
    ar = np.zeros((p.nx, p.ny))
    hm = np.zeros((p.nx, p.ny))
    for i in range(p.nx):
        for j in range(p.ny):
            mem = bf.box_members(comp, i, j, p.sub)
            vals = np.array([bf._ext(e, a, b, p.bc) for a, b, _ in mem])
            wts = np.array([w for _, _, w in mem])
            ar[i, j] = np.sum(wts * vals)
            hm[i, j] = 1.0 / np.sum(wts / vals)
    return ar, hm


@pytest.mark.parametrize("axis", [0, 1])
@pytest.mark.parametrize("edge", [7, 10])
def test_grid_aligned_flat_interface_gives_exact_means(axis, edge):
    # A step in C along `axis`: the interface normal is exactly that axis, so
    # the field component across it sees the harmonic mean and the others the
    # arithmetic mean of the subpixel permittivity (Eq. 7 limits).
    n = 24
    C = np.zeros((n, n))
    if axis == 0:
        C[edge:, :] = 1.0
    else:
        C[:, edge:] = 1.0
    p = prob(mx=n, my=n, radius=3.0, beta=8.0, bc=CLAMP)
    fw = orc.forward(p, C)
    e = fw["e"]
    k = p.k0 + 1
    ex, ey, ez = fw["eps_hat"][0, :, :, k], fw["eps_hat"][1, :, :, k], fw["eps_hat"][2, :, :, k]
    ar_x, hm_x = _box_means(e, 0, p)
    ar_y, hm_y = _box_means(e, 1, p)
    ar_z, _ = _box_means(e, 2, p)
    across, along = (ex, ey) if axis == 0 else (ey, ex)
    hm_across = hm_x if axis == 0 else hm_y
    ar_along = ar_y if axis == 0 else ar_x
    np.testing.assert_allclose(across, hm_across, rtol=1e-13)
    np.testing.assert_allclose(along, ar_along, rtol=1e-13)
    np.testing.assert_allclose(ez, ar_z, rtol=1e-13)
    # and the interface really is resolved (harmonic < arithmetic somewhere)
    ar_across = ar_x if axis == 0 else ar_y
    assert np.max(ar_across - hm_across) > 1e-2


def test_diagonal_interface_takes_half_and_half():
    # 45-degree linear ramp: m = 1/2, so eps = 1 / (H/2 + 1/(2A)).
    n = 20
    a = np.arange(n)[:, None]
    b = np.arange(n)[None, :]
    C = 0.3 + 0.02 * (a + b)
    p = prob(mx=n, my=n, radius=0.5, beta=8.0)
    fw = orc.forward(p, C)
    inner = (slice(2, p.nx - 2), slice(2, p.ny - 2))
    for c in range(2):
        ref = 1.0 / (0.5 * fw["H"][c] + 0.5 / fw["A"][c])
        np.testing.assert_allclose(fw["eps_c"][c][inner], ref[inner], rtol=1e-13)


def test_offdiagonal_flat_and_diagonal():
    n = 20
    a = np.arange(n)[:, None]
    b = np.arange(n)[None, :]
    p = prob(mx=n, my=n, radius=0.5, beta=8.0)
    C = 0.3 + 0.02 * a + 0 * b                     # normal along x: n_x n_y = 0
    od = orc.forward(p, C, offdiag=True)["offdiag"]
    np.testing.assert_allclose(od[:, 2:-2, 2:-2, p.k0 + 1], 0.0, atol=1e-15)
    C = 0.3 + 0.02 * (a + b)                       # 45 degrees: n_x n_y = 1/2
    fw = orc.forward(p, C, offdiag=True)
    for c in range(2):
        ref = 0.5 * (fw["H"][c] - 1.0 / fw["A"][c])
        np.testing.assert_allclose(fw["offdiag"][c, 2:-2, 2:-2, p.k0 + 1], ref[2:-2, 2:-2],
                                   rtol=1e-12, atol=1e-15)
    C = 0.3 + 0.02 * (a - b)                       # -45 degrees: n_x n_y = -1/2
    fw = orc.forward(p, C, offdiag=True)
    ref = -0.5 * (fw["H"][0] - 1.0 / fw["A"][0])
    np.testing.assert_allclose(fw["offdiag"][0, 2:-2, 2:-2, p.k0 + 1], ref[2:-2, 2:-2],
                               rtol=1e-12, atol=1e-15)


def test_harmonic_never_exceeds_arithmetic():
    rng = np.random.default_rng(6)
    p = prob(mx=32, my=32, radius=3.0, beta=16.0)
    fw = orc.forward(p, rng.random((32, 32)))
    for c in range(2):
        e = fw["eps_c"][c]
        assert np.all(e <= fw["A"][c] * (1 + 1e-14))
        assert np.all(e >= 1.0 / fw["H"][c] * (1 - 1e-14))


# --------------------------------------------------------------- VJP (Eq. 1)

def _complex_step_jacobian(p, C, h=1e-30):
    n = C.size
    J = np.zeros((3 * p.nx * p.ny * p.nz, n))
    for idx in range(n):
        Cc = C.astype(np.complex128)
        Cc.flat[idx] += 1j * h
        J[:, idx] = np.imag(orc.eps_hat(p, Cc)).ravel() / h
    return J


@pytest.mark.parametrize("bc", [CLAMP, PERIODIC])
@pytest.mark.parametrize("radius,beta", [(2.0, 8.0), (3.0, 32.0)])
def test_vjp_matches_complex_step_jacobian(bc, radius, beta):
    rng = np.random.default_rng(7)
    p = prob(mx=8, my=8, nz=14, radius=radius, beta=beta, bc=bc)
    C = 0.5 + 0.25 * rng.standard_normal((8, 8))
    J = _complex_step_jacobian(p, C)
    assert np.abs(J).max() > 1.0
    for _ in range(2):
        G = rng.standard_normal((3, p.nx, p.ny, p.nz))
        ref = (J.T @ G.ravel()).reshape(8, 8)
        got = orc.vjp_real(p, C, G)
        np.testing.assert_allclose(got, ref, rtol=1e-10, atol=1e-10 * np.abs(ref).max())


def test_vjp_fields_is_minus_two_re_of_field_product():
    rng = np.random.default_rng(8)
    p = prob(mx=8, my=8, nz=14, radius=2.0, beta=8.0)
    C = rng.random((8, 8))
    shape = (3, p.nx, p.ny, p.nz)
    EF = [rng.standard_normal(shape) + 1j * rng.standard_normal(shape) for _ in range(2)]
    EA = [rng.standard_normal(shape) + 1j * rng.standard_normal(shape) for _ in range(2)]
    J = _complex_step_jacobian(p, C)
    w = sum((ef * ea) for ef, ea in zip(EF, EA))     # unconjugated product
    ref = (-2.0 * (J.T @ w.ravel()).real).reshape(8, 8)
    got = orc.vjp_fields(p, C, EF, EA)
    np.testing.assert_allclose(got, ref, rtol=1e-10, atol=1e-10 * np.abs(ref).max())
    # wavelengths add
    one = orc.vjp_fields(p, C, EF[:1], EA[:1]) + orc.vjp_fields(p, C, EF[1:], EA[1:])
    np.testing.assert_allclose(got, one, rtol=1e-12, atol=1e-12)


def test_vjp_central_finite_differences_cfg1():
    from paper_2505_03352_gb300 import synth
    w = synth.WORKLOADS[1]
    p = orc.Problem(mx=w.mx, my=w.my, nz=w.nz, radius=w.radius, beta=w.beta)
    C = synth.controls(w).astype(np.float64)
    EF, EA = synth.fields(w)
    G = orc.field_cotangent(p, EF, EA)
    grad = orc.vjp_real(p, C, G)
    rng = np.random.default_rng(9)
    h = 1e-6
    for idx in rng.choice(C.size, 12, replace=False):
        Cp, Cm = C.copy(), C.copy()
        Cp.flat[idx] += h
        Cm.flat[idx] -= h
        fd = (np.sum(G * orc.eps_hat(p, Cp)) - np.sum(G * orc.eps_hat(p, Cm))) / (2 * h)
        assert abs(fd - grad.flat[idx]) <= 1e-6 * max(1.0, np.abs(grad).max())


def test_vjp_uniform_design_semi_closed_form():
    # Periodic, uniform C and uniform cotangent g on every plane:
    # dJ/dC = P'(c) (eps_core - eps_clad) g [(3 nk - 1)/4 + eps_f^2 / (4 e^2)].
    c, g = 0.47, 0.8
    p = prob(mx=12, my=12, nz=16, radius=3.0, beta=16.0, bc=PERIODIC)
    C = np.full((12, 12), c)
    G = np.full((3, p.nx, p.ny, p.nz), g)
    got = orc.vjp_real(p, C, G)
    t = np.tanh(16.0 * (c - 0.5))
    rho = 0.5 * (1 + t)
    e = 2.085 + rho * (12.11 - 2.085)
    ef = 1.0 / (0.5 / e + 0.5 / 2.085)
    ref = 8.0 * (1 - t * t) * (12.11 - 2.085) * g * ((3 * 11 - 1) / 4 + ef ** 2 / (4 * e ** 2))
    np.testing.assert_allclose(got, ref, rtol=1e-13)


def test_vjp_ignores_cladding_planes():
    rng = np.random.default_rng(10)
    p = prob(mx=8, my=8, nz=16, radius=2.0, beta=8.0)
    C = rng.random((8, 8))
    G = rng.standard_normal((3, p.nx, p.ny, p.nz))
    k0, nk = p.k0, p.slab_nk
    G[0, :, :, k0 + 1:k0 + nk + 1] = 0
    G[1, :, :, k0 + 1:k0 + nk + 1] = 0
    G[2, :, :, k0:k0 + nk + 1] = 0
    assert np.all(orc.vjp_real(p, C, G) == 0)
