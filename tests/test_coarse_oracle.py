"""Pins of the coarse-control oracle (Eq. 2 on a node grid): partition of
unity, exact reproduction of linear functions, the double sum written out
node by node, the transpose, and complex-step / finite-difference
derivatives of the whole chain with respect to the node values."""

import numpy as np
import pytest

from oracle import coarse_oracle as co
from oracle import epschain_oracle as orc


def test_expansion_is_the_double_sum():
    rng = np.random.default_rng(1)
    c = rng.standard_normal((5, 4))
    mx, my = 14, 10
    hx, hy = mx / 4, my / 3
    phi = np.zeros((mx, my))
    for a in range(mx):
        for b in range(my):
            for i in range(5):
                for j in range(4):
                    bx = max(0.0, 1 - abs((a + 0.5 - i * hx) / hx))
                    by = max(0.0, 1 - abs((b + 0.5 - j * hy) / hy))
                    phi[a, b] += c[i, j] * bx * by
    np.testing.assert_allclose(co.expand(c, mx, my), phi, rtol=0, atol=1e-14)


@pytest.mark.parametrize("m,nc", [(420, 36), (64, 5), (30, 2), (17 * 2, 9)])
def test_partition_of_unity(m, nc):
    np.testing.assert_allclose(co.basis_matrix(m, nc).sum(axis=1), 1.0, rtol=0, atol=1e-14)


def test_linear_functions_are_reproduced():
    # c_ij = alpha X_i + gamma Y_j + delta gives Phi = alpha x + gamma y + delta
    mx, my, ncx, ncy = 420, 96, 36, 9
    hx, hy = mx / (ncx - 1), my / (ncy - 1)
    X = np.arange(ncx) * hx
    Y = np.arange(ncy) * hy
    c = 0.01 * X[:, None] - 0.03 * Y[None, :] + 0.4
    x = np.arange(mx) + 0.5
    y = np.arange(my) + 0.5
    ref = 0.01 * x[:, None] - 0.03 * y[None, :] + 0.4
    np.testing.assert_allclose(co.expand(c, mx, my), ref, rtol=0, atol=1e-12)


def test_paper_layout_has_integer_stride_and_two_nodes_per_axis():
    B = co.basis_matrix(420, 36)          # 210 Yee cells x 2 subpixels, 36 controls
    assert np.all((B > 0).sum(axis=1) == 2)
    assert 420 / 35 == 12


def test_transpose_is_adjoint():
    rng = np.random.default_rng(2)
    c = rng.standard_normal((6, 7))
    g = rng.standard_normal((40, 36))
    lhs = np.sum(co.expand(c, 40, 36) * g)
    rhs = np.sum(c * co.expand_T(g, 6, 7))
    assert abs(lhs - rhs) < 1e-12 * max(1.0, abs(lhs))


@pytest.mark.parametrize("bc", [orc.CLAMP, orc.PERIODIC])
def test_chain_vjp_matches_complex_step(bc):
    rng = np.random.default_rng(3)
    p = orc.Problem(mx=16, my=12, nz=14, radius=3.0, beta=8.0, bc=bc)
    c = 0.5 + 0.3 * rng.standard_normal((5, 4))
    h = 1e-30
    J = np.zeros((3 * p.nx * p.ny * p.nz, c.size))
    for i in range(c.size):
        z = c.astype(np.complex128)
        z.flat[i] += 1j * h
        J[:, i] = np.imag(co.eps_hat_coarse(p, z)).ravel() / h
    assert np.abs(J).max() > 0.1
    G = rng.standard_normal((3, p.nx, p.ny, p.nz))
    ref = (J.T @ G.ravel()).reshape(c.shape)
    np.testing.assert_allclose(co.vjp_real_coarse(p, c, G), ref, rtol=1e-10,
                               atol=1e-10 * np.abs(ref).max())


def test_chain_vjp_central_finite_differences():
    rng = np.random.default_rng(4)
    p = orc.Problem(mx=48, my=40, nz=16, radius=3.0, beta=8.0)
    c = 0.5 + 0.3 * rng.standard_normal((9, 6))
    shape = (3, p.nx, p.ny, p.nz)
    EF = [rng.standard_normal(shape) + 1j * rng.standard_normal(shape)]
    EA = [rng.standard_normal(shape) + 1j * rng.standard_normal(shape)]
    G = orc.field_cotangent(p, EF, EA)
    grad = co.vjp_fields_coarse(p, c, EF, EA)
    hstep = 1e-6
    for idx in range(c.size):
        cp, cm = c.copy(), c.copy()
        cp.flat[idx] += hstep
        cm.flat[idx] -= hstep
        fd = (np.sum(G * co.eps_hat_coarse(p, cp)) - np.sum(G * co.eps_hat_coarse(p, cm))) / (2 * hstep)
        assert abs(fd - grad.flat[idx]) <= 1e-6 * max(1.0, np.abs(grad).max())


def test_uniform_nodes_give_the_uniform_design():
    p = orc.Problem(mx=24, my=24, nz=16, radius=3.0, beta=8.0, bc=orc.PERIODIC)
    c = np.full((4, 5), 0.62)
    rho = 0.5 * (1 + np.tanh(8.0 * (0.62 - 0.5)))
    e = p.eps_clad + rho * (p.eps_core - p.eps_clad)
    eh = co.eps_hat_coarse(p, c)
    lo, hi = orc.support_planes(p)["xy"]
    np.testing.assert_allclose(eh[0, :, :, lo:hi], e, rtol=1e-13)
