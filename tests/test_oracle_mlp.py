"""Pins of the MLP oracle: analytic gradients against central finite
differences in FP64, the GELU closed forms, a hand-computed Adam step, and the
bfloat16 rounding rule."""
import math

import numpy as np

from oracle import mlp


def test_parameter_count():
    assert mlp.N_PARAMS == 9348


def test_gelu_values_and_derivative():
    x = np.array([-3.0, -1.0, 0.0, 0.5, 2.0])
    # x * Phi(x) with Phi from math.erfc (independent of the erf path)
    phi = np.array([0.5 * math.erfc(-t / math.sqrt(2)) for t in x])
    np.testing.assert_allclose(mlp.gelu(x), x * phi, rtol=1e-14, atol=1e-16)
    h = 1e-6
    fd = (mlp.gelu(x + h) - mlp.gelu(x - h)) / (2 * h)
    np.testing.assert_allclose(mlp.gelu_grad(x), fd, rtol=1e-8, atol=1e-9)


def test_gradient_against_finite_differences():
    rng = np.random.default_rng(3)
    theta = mlp.init_params(1) + 0.01 * rng.standard_normal(mlp.N_PARAMS)
    X = rng.standard_normal((16, 76))
    Y = rng.standard_normal((16, 4))
    g = mlp.grad(theta, X, Y)
    idx = rng.choice(mlp.N_PARAMS, 60, replace=False)
    # include every bias block and the last layer
    idx = np.concatenate([idx, [64 * 76, 64 * 76 + 63, 9348 - 1, 9348 - 5, 9348 - 10]])
    h = 1e-6
    for k in idx:
        e = np.zeros_like(theta)
        e[k] = h
        fd = (mlp.loss(theta + e, X, Y) - mlp.loss(theta - e, X, Y)) / (2 * h)
        assert abs(fd - g[k]) <= 1e-7 * max(1.0, abs(g[k])), (k, fd, g[k])


def test_adam_first_step_closed_form():
    """At t = 1 with zero moments the bias-corrected step is lr * g / (|g| + eps)."""
    g = np.array([0.3, -2.0, 1e-3])
    th, m, v = mlp.adam_step(np.zeros(3), g, np.zeros(3), np.zeros(3), 1, lr=0.01)
    np.testing.assert_allclose(th, -0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12)
    np.testing.assert_allclose(m, 0.1 * g)
    np.testing.assert_allclose(v, 0.001 * g * g)


def test_bf16_rounding():
    x = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, -3.14159265, 1e-20])
    r = mlp.to_bf16(x)
    assert r[0] == 1.0
    assert r[1] == 1.0  # halfway, ties to even
    assert r[2] == 1.0 + 2 ** -7  # above halfway rounds up
    assert abs(r[3] - (-3.140625)) < 1e-12
    # 8 significant bits
    m, _ = np.frexp(r[4])
    assert np.all((m * 2 ** 8) == np.round(m * 2 ** 8))
