"""Randomised properties of the FP64 oracle over shapes the fixed pins do
not reach: ragged and non-square regions, radii from below one subpixel to
5, slabs anywhere in z (including against the top and bottom planes), beta
up to 32 and both boundary rules.

- Adjoint identity: <vjp_real(G), v> = <G, J v>, with J v the complex-step
  directional derivative of eps_hat (exact to rounding, no step error).
- Eq. 1 form: vjp_fields equals -2 Re of vjp_real applied to the summed,
  unconjugated field product (real and imaginary parts by linearity).
- Forward bounds: every eps_hat entry lies between eps_clad and eps_core.
- Filter: under the periodic rule the sum of u equals the sum of C.
- The same adjoint identity for the morphology chain (random alpha, disk
  radius and dilate/erode sequences) and for coarse control nodes (random
  node grids).
- 3-D face normals: the face rows are those of a unit-normal tensor, and
  every other plane equals the base chain's.
- Adam (Eq. 10-11) with a zero stabiliser: scaling every gradient of a
  multi-step run by a power of two leaves the trajectory bit for bit (the
  update depends on M / sqrt(V) only), and negating the gradients negates
  the update from a zero design.

The examples are drawn by hypothesis when it is installed."""

import numpy as np
import pytest

from oracle import epschain_oracle as orc

hyp = pytest.importorskip("hypothesis")
st = hyp.strategies
given, settings = hyp.given, hyp.settings


@st.composite
def problems(draw):
    mx = 2 * draw(st.integers(2, 7))
    my = 2 * draw(st.integers(2, 7))
    nz = draw(st.integers(3, 10))
    nk = draw(st.integers(1, nz - 2))
    k0 = draw(st.integers(0, nz - 1 - nk))
    radius = draw(st.sampled_from([0.5, 1.0, 1.5, 2.0, 2.5, 3.0, 4.0, 5.0]))
    beta = draw(st.sampled_from([1.0, 4.0, 8.0, 16.0, 32.0]))
    eta = draw(st.sampled_from([0.3, 0.5, 0.7]))
    bc = draw(st.sampled_from([orc.CLAMP, orc.PERIODIC]))
    seed = draw(st.integers(0, 2 ** 31 - 1))
    p = orc.Problem(mx=mx, my=my, nz=nz, radius=radius, beta=beta, eta=eta, bc=bc,
                    slab_k0=k0, slab_nk=nk)
    return p, np.random.default_rng(seed)


def _jvp(p, C, v, h=1e-30):
    return np.imag(orc.eps_hat(p, C.astype(np.complex128) + 1j * h * v)) / h


@settings(max_examples=40, deadline=None)
@given(problems())
def test_vjp_real_is_the_adjoint_of_the_forward_derivative(case):
    p, rng = case
    C = rng.random((p.mx, p.my))
    v = rng.standard_normal((p.mx, p.my))
    G = rng.standard_normal((3, p.nx, p.ny, p.nz))
    lhs = float(np.sum(orc.vjp_real(p, C, G) * v))
    rhs = float(np.sum(G * _jvp(p, C, v)))
    assert lhs == pytest.approx(rhs, rel=1e-9, abs=1e-12 * (1 + abs(rhs)))


@settings(max_examples=25, deadline=None)
@given(problems(), st.integers(1, 3))
def test_eq1_form_is_minus_two_re_of_the_real_vjp(case, n_lambda):
    p, rng = case
    C = rng.random((p.mx, p.my))
    shape = (3, p.nx, p.ny, p.nz)
    EF = [rng.standard_normal(shape) + 1j * rng.standard_normal(shape) for _ in range(n_lambda)]
    EA = [rng.standard_normal(shape) + 1j * rng.standard_normal(shape) for _ in range(n_lambda)]
    w = sum(ef * ea for ef, ea in zip(EF, EA))
    ref = -2.0 * orc.vjp_real(p, C, np.real(w))
    got = orc.vjp_fields(p, C, EF, EA)
    np.testing.assert_allclose(got, ref, rtol=1e-10, atol=1e-10 * (1 + np.abs(ref).max()))


@settings(max_examples=40, deadline=None)
@given(problems())
def test_eps_hat_lies_between_the_two_materials(case):
    p, rng = case
    C = rng.random((p.mx, p.my))
    e = orc.eps_hat(p, C)
    assert np.all(e >= p.eps_clad * (1 - 1e-12)) and np.all(e <= p.eps_core * (1 + 1e-12))


@settings(max_examples=30, deadline=None)
@given(problems())
def test_periodic_filter_preserves_the_sum(case):
    p, rng = case
    q = orc.Problem(mx=p.mx, my=p.my, nz=p.nz, radius=p.radius, beta=p.beta, bc=orc.PERIODIC,
                    slab_k0=p.slab_k0, slab_nk=p.slab_nk)
    C = rng.random((p.mx, p.my))
    u = orc.forward(q, C)["u"]
    assert float(u.sum()) == pytest.approx(float(C.sum()), rel=1e-12)


@st.composite
def morphs(draw):
    from oracle import morph_oracle as mo
    alpha = draw(st.sampled_from([5.0, 20.0, 60.0]))
    radius = draw(st.sampled_from([0.0, 0.5, 1.0, 1.5, 2.0, 2.5]))
    ops = tuple(draw(st.lists(st.sampled_from([mo.DILATE, mo.ERODE]), min_size=0, max_size=4)))
    return mo.Morph(alpha=alpha, radius=radius, ops=ops)


@settings(max_examples=25, deadline=None)
@given(problems(), morphs())
def test_morphology_vjp_is_the_adjoint_of_its_forward_derivative(case, morph):
    from oracle import morph_oracle as mo
    p, rng = case
    C = rng.random((p.mx, p.my))
    v = rng.standard_normal((p.mx, p.my))
    G = rng.standard_normal((3, p.nx, p.ny, p.nz))
    h = 1e-30
    jv = np.imag(mo.eps_hat_morph(p, morph, C.astype(np.complex128) + 1j * h * v)) / h
    lhs = float(np.sum(mo.vjp_real_morph(p, morph, C, G) * v))
    rhs = float(np.sum(G * jv))
    assert lhs == pytest.approx(rhs, rel=1e-8, abs=1e-12 * (1 + abs(rhs)))


@settings(max_examples=25, deadline=None)
@given(problems(), st.integers(2, 6), st.integers(2, 6))
def test_coarse_vjp_is_the_adjoint_of_its_forward_derivative(case, ncx, ncy):
    from oracle import coarse_oracle as co
    p, rng = case
    c = rng.random((ncx, ncy))
    v = rng.standard_normal((ncx, ncy))
    G = rng.standard_normal((3, p.nx, p.ny, p.nz))
    h = 1e-30
    jv = np.imag(co.eps_hat_coarse(p, c.astype(np.complex128) + 1j * h * v)) / h
    lhs = float(np.sum(co.vjp_real_coarse(p, c, G) * v))
    rhs = float(np.sum(G * jv))
    assert lhs == pytest.approx(rhs, rel=1e-9, abs=1e-12 * (1 + abs(rhs)))


@settings(max_examples=25, deadline=None)
@given(problems())
def test_face_rows_are_those_of_a_unit_normal_tensor(case):
    # 3-D face normals: on each face plane, row z of T = (a - b) n n^T + b I
    # with |n| = 1 obeys (T_zz - b)(a - b) = T_zx^2 + T_zy^2 + (T_zz - b)^2,
    # with T_zz between a and b; other planes equal the base chain's.  a - b
    # is a difference of O(1) numbers, so near-binary pixels (large beta)
    # carry a few ulps of max(|a|, |b|, |T_zz|) of absolute error in a - b and
    # T_zz - b; the identity then holds to that times (|T_zz - b| + |a - b|),
    # while a dropped or mis-signed term leaves an error of order
    # |T_zz - b| |a - b|.
    from oracle import normals3d_oracle as n3
    p, rng = case
    C = rng.random((p.mx, p.my))
    eps, od = n3.forward_3d(p, C)
    fw = orc.forward(p, C, offdiag=True)
    a = 0.5 * (fw["H"][2] + 1 / p.eps_clad)
    b = 1 / (0.5 * (fw["A"][2] + p.eps_clad))
    faces = [p.k0, p.k0 + p.slab_nk]
    for k in faces:
        t = 1 / eps[2, :, :, k] - b
        lhs = t * (a - b)
        rhs = od[2, :, :, k] ** 2 + od[3, :, :, k] ** 2 + t * t
        m = np.maximum(np.maximum(np.abs(a), np.abs(b)), np.abs(1 / eps[2, :, :, k]))
        tol = 64 * np.finfo(float).eps * m * (np.abs(t) + np.abs(a - b))
        assert np.all(np.abs(lhs - rhs) <= tol + 1e-300)
        lo, hi = np.minimum(a, b), np.maximum(a, b)
        te = 1 / eps[2, :, :, k]
        assert np.all(te >= lo * (1 - 1e-12)) and np.all(te <= hi * (1 + 1e-12))
    mask = np.ones(p.nz, bool)
    mask[faces] = False
    np.testing.assert_array_equal(eps[:2], fw["eps_hat"][:2])
    np.testing.assert_array_equal(eps[2][..., mask], fw["eps_hat"][2][..., mask])


@st.composite
def adam_runs(draw):
    steps = draw(st.integers(1, 8))
    shape = (draw(st.integers(1, 6)), draw(st.integers(1, 6)))
    b1 = draw(st.sampled_from([0.0, 0.5, 0.9]))
    b2 = draw(st.sampled_from([0.9, 0.99, 0.999]))
    k = draw(st.integers(-20, 20))
    seed = draw(st.integers(0, 2 ** 31 - 1))
    rng = np.random.default_rng(seed)
    G = [rng.standard_normal(shape) * 10.0 ** rng.integers(-4, 4, shape) for _ in range(steps)]
    return b1, b2, k, G, rng.random(shape)


def _adam_trajectory(p, C, G):
    from oracle import optimizer_oracle as oo
    M = np.zeros_like(C)
    V = np.zeros_like(C)
    out = []
    for i, g in enumerate(G, start=1):
        C, M, V = oo.adam_update(C, g, M, V, i, p)
        out.append(C)
    return out


@settings(max_examples=60, deadline=None)
@given(adam_runs())
def test_adam_step_is_invariant_to_gradient_scale_and_odd_in_its_sign(run):
    from oracle import optimizer_oracle as oo
    b1, b2, k, G, C0 = run
    p = oo.OptParams(b1=b1, b2=b2, adam_eps=0.0)
    base = _adam_trajectory(p, C0, G)
    scaled = _adam_trajectory(p, C0, [np.ldexp(g, k) for g in G])
    for a, b in zip(base, scaled):
        np.testing.assert_array_equal(a, b)
    zero = np.zeros_like(C0)
    pos = _adam_trajectory(p, zero, G)
    neg = _adam_trajectory(p, zero, [-g for g in G])
    for a, b in zip(pos, neg):
        np.testing.assert_array_equal(a, -b)
