"""Pins of the optimiser oracle (Eq. 10-15) to closed forms: Adam's
sign-like first step and constant-gradient steps, the schedule's end points
and monotonicity, the fixed point of the beta_max control under the model
u = 1/(1 + k beta) that Eq. 15 inverts, and a brute-force gray count."""

import numpy as np
import pytest

from oracle import optimizer_oracle as oo


def test_first_adam_step_moves_each_control_by_lr_times_sign():
    # M^ = G and V^ = G^2 after one step: the update is lr G / (|G| + eps)
    rng = np.random.default_rng(1)
    G = rng.standard_normal((7, 9)) * 10.0 ** rng.integers(-3, 3, (7, 9))
    C = rng.random((7, 9))
    p = oo.OptParams(lr=0.01, adam_eps=0.0)
    C1, M, V = oo.adam_update(C, G, np.zeros_like(G), np.zeros_like(G), 1, p)
    np.testing.assert_allclose(C1, C - 0.01 * np.sign(G), rtol=0, atol=1e-15)
    np.testing.assert_allclose(M, 0.1 * G, rtol=1e-15)
    np.testing.assert_allclose(V, 0.001 * G * G, rtol=1e-12)


def test_constant_gradient_keeps_unit_normalised_steps():
    # with a constant gradient the bias-corrected moments equal G and G^2
    # exactly at every step, so each step is again lr * sign(G)
    G = np.array([[2.0, -0.5], [1e-3, -7.0]])
    C = np.zeros_like(G)
    M = np.zeros_like(G)
    V = np.zeros_like(G)
    p = oo.OptParams(lr=0.02, adam_eps=0.0)
    for i in range(1, 30):
        C, M, V = oo.adam_update(C, G, M, V, i, p)
        np.testing.assert_allclose(C, -0.02 * i * np.sign(G), rtol=1e-12)


def test_beta_schedule_end_points_and_monotone():
    assert oo.beta_schedule(0, 100, 10.0, 200.0) == 10.0
    assert abs(oo.beta_schedule(100, 100, 10.0, 200.0) - 200.0) < 1e-12
    b = [oo.beta_schedule(i, 100, 10.0, 200.0) for i in range(101)]
    assert all(x < y for x, y in zip(b, b[1:]))
    # halfway: (exp(1/4) - 1) / (e - 1) of the way
    mid = 10.0 + 190.0 * (np.exp(0.25) - 1) / (np.e - 1)
    assert abs(oo.beta_schedule(50, 100, 10.0, 200.0) - mid) < 1e-12


def test_beta_max_control_fixed_point():
    # if u = 1 / (1 + k beta) then (1/u - 1)/beta = k for every beta, t -> k
    # and beta_max -> (1/u0 - 1) / k: the beta at which u would equal u0
    k, u0, gamma = 0.37, 0.01, 0.95
    t, beta_max = 0.0, 50.0
    for beta in np.linspace(10, 80, 400):
        u = 1.0 / (1.0 + k * beta)
        t, beta_max = oo.beta_max_control(t, beta_max, u, beta, gamma, u0)
    assert abs(t - k) < 1e-12
    target = (1 / u0 - 1) / k
    assert abs(beta_max - target) < 1e-6 * target
    assert abs(1.0 / (1.0 + k * beta_max) - u0) < 1e-8


def test_first_sample_initialises_t():
    t, bm = oo.beta_max_control(0.0, 100.0, 0.2, 10.0, 0.95, 0.01)
    assert t == pytest.approx((1 / 0.2 - 1) / 10.0)
    assert bm == pytest.approx(0.95 * 100.0 + 0.05 * 99.0 / t)


def test_gray_count_brute_force():
    rng = np.random.default_rng(2)
    rho = rng.random((13, 11))
    rho[0, :3] = [0.05, 0.95, 0.0500001]
    n = 0
    for v in rho.ravel():
        if 0.05 < v < 0.95:
            n += 1
    assert oo.gray_count(rho, 0.05) == n


def test_opt_step_order_and_floor():
    p = oo.OptParams(n_iter=10)
    s = oo.init_state(p)
    assert s.beta == pytest.approx(oo.beta_schedule(1, 10, 10.0, 100.0))
    rho = np.zeros((4, 4))                 # binary design: u floored at one pixel
    C = np.zeros((4, 4))
    G = np.ones((4, 4))
    C1, M, V, s1 = oo.opt_step(p, s, C, G, np.zeros_like(C), np.zeros_like(C), rho)
    assert s1.step == 1 and s1.gray == 0 and s1.unbinarity == pytest.approx(1 / 16)
    assert s1.t == pytest.approx(15.0 / s.beta)
    assert s1.beta == pytest.approx(oo.beta_schedule(2, 10, 10.0, s1.beta_max))
    np.testing.assert_allclose(C1, -p.lr * 1.0 / (1.0 + p.adam_eps), rtol=1e-12)
