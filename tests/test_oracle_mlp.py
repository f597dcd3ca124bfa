"""Pins of the FP64 reference network used to check the GPU training kernels."""
import math

import numpy as np

from oracle import mlp


def test_gelu_matches_erf_definition():
    xs = np.linspace(-6, 6, 97)
    ref = np.array([0.5 * x * (1 + math.erf(x / math.sqrt(2))) for x in xs])
    np.testing.assert_allclose(mlp.gelu(xs), ref, rtol=1e-14, atol=1e-14)
    h = 1e-6
    fd = (mlp.gelu(xs + h) - mlp.gelu(xs - h)) / (2 * h)
    np.testing.assert_allclose(mlp.gelu_grad(xs), fd, rtol=1e-7, atol=1e-8)


def test_parameter_count():
    assert mlp.N_PARAMS == 5 * 64 + 64 + 64 * 64 + 64 + 64 * 64 + 64 + 64 * 3 + 3


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(3)
    p = mlp.init_params(1).astype(np.float64)
    X = rng.standard_normal((17, 5))
    T = rng.standard_normal((17, 3))
    _, g = mlp.loss_and_grad(p, X, T)
    idx = rng.choice(p.size, size=60, replace=False)
    h = 1e-6
    for i in idx:
        e = np.zeros_like(p)
        e[i] = h
        fd = (mlp.loss_and_grad(p + e, X, T)[0] - mlp.loss_and_grad(p - e, X, T)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), i


def test_bf16_rounding():
    vals = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 2 ** -7, -3.14159, 1e-20], dtype=np.float32)
    r = mlp.bf16_round(vals)
    assert r[0] == 1.0
    assert r[1] == 1.0                 # tie rounds to even
    assert r[2] == 1.0 + 2 ** -7       # representable
    assert abs(r[3] + 3.14159) < 2 ** -7 * 4
    assert r[4] != 0


def test_first_adam_step_moves_by_lr_sign():
    # bias correction makes m_hat = g and v_hat = g^2 on the first step
    rng = np.random.default_rng(5)
    p = rng.standard_normal(50)
    g = rng.standard_normal(50)
    new, m, v = mlp.adam_step(p, g, np.zeros(50), np.zeros(50), 1, lr=1e-3)
    np.testing.assert_allclose(new, p - 1e-3 * np.sign(g) * np.abs(g) / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)
    np.testing.assert_allclose(m, 0.1 * g)
    np.testing.assert_allclose(v, 0.001 * g * g)


def test_features_hand_worked_row():
    # shell 1: P0 = 300, P_SN = 100 -> D = 400; k = 0.4 with k_N = 0.8
    idx, X, T = mlp.features_and_targets(
        k_mean=[0.1, 0.4, 0.5, 0.6], n_modes=[0, 12, 8, 4], p0=[1.0, 300.0, -150.0, np.nan],
        p2=[0.0, 40.0, 1.0, 1.0], p4=[0.0, -20.0, 1.0, 1.0], p_sn=100.0, k_nyq=0.8,
        fine=([0.0, 340.0, 0.0, 0.0], [0.0, 44.0, 0.0, 0.0], [0.0, -22.0, 0.0, 0.0]))
    # shell 0 has no modes, shell 2 has D = -50 <= 0, shell 3 is not finite
    assert list(idx) == [1]
    np.testing.assert_allclose(X[0], [0.5, math.log(4.0), 0.1, -0.05, 0.25], rtol=1e-15)
    np.testing.assert_allclose(T[0], [0.1, 0.01, -0.005], rtol=1e-13)
