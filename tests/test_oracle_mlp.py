"""Pins of the FP64 MLP oracle: gradients against central differences, GELU
against its definition through a library CDF, Adam against its closed form."""
import math

import numpy as np
from scipy.stats import norm

from oracle import mlp


def test_gelu_is_z_times_normal_cdf():
    z = np.linspace(-6, 6, 101)
    assert np.allclose(mlp.gelu(z), z * norm.cdf(z), rtol=1e-14, atol=1e-15)
    h = 1e-6
    assert np.allclose(mlp.gelu_grad(z), (mlp.gelu(z + h) - mlp.gelu(z - h)) / (2 * h), rtol=1e-8, atol=1e-9)


def test_parameter_layout():
    assert mlp.n_params() == 256 * 64 + 256 + 256 * 256 + 256 + 2 * 256 + 2
    theta = mlp.init_params(0)
    assert np.array_equal(mlp.pack(mlp.unpack(theta)), theta)
    p = mlp.unpack(theta)
    assert np.abs(p["W1"]).max() <= math.sqrt(6 / 64) and np.all(p["b2"] == 0)


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(1)
    theta = mlp.init_params(3) + 0.01 * rng.standard_normal(mlp.n_params())
    X = rng.standard_normal((5, 64))
    T = rng.standard_normal((5, 2))
    g = mlp.gradient(theta, X, T)
    idx = rng.choice(mlp.n_params(), 60, replace=False)
    h = 1e-6
    for i in idx:
        e = np.zeros_like(theta)
        e[i] = h
        fd = (mlp.loss(theta + e, X, T) - mlp.loss(theta - e, X, T)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])) + 1e-9, (i, fd, g[i])


def test_adam_first_step_is_lr_times_sign():
    """With m = v = 0, the first Adam step moves each parameter by
    lr * g / (|g| + eps / sqrt(1 - b2)) ~ lr * sign(g)."""
    g = np.array([0.3, -2.0, 1e-3])
    th, m, v = mlp.adam_step(np.zeros(3), np.zeros(3), np.zeros(3), g, 1, lr=0.01)
    expect = -0.01 * g / (np.abs(g) + 1e-8)
    assert np.allclose(th, expect, rtol=1e-12)


def test_adam_constant_gradient_moves_by_lr_every_step():
    """With a constant gradient g, m_t = (1 - b1^t) g and v_t = (1 - b2^t) g^2,
    so the bias-corrected moments are exactly g and g^2 at every step and each
    step moves by lr * g / (|g| + eps).  A wrong power of b1 or b2 in the
    bias correction breaks this from the second step on (the first step hides
    it: there m_hat = g and v_hat = g^2 whatever the exponent)."""
    g = np.array([0.3, -2.0, 1e-3, 5.0])
    th, m, v = np.zeros(4), np.zeros(4), np.zeros(4)
    step = -0.01 * g / (np.abs(g) + 1e-8)
    for t in range(1, 11):
        prev = th
        th, m, v = mlp.adam_step(th, m, v, g, t, lr=0.01)
        assert np.allclose(th - prev, step, rtol=1e-9, atol=0.0), t
        assert np.allclose(m, (1 - 0.9 ** t) * g, rtol=1e-12)
        assert np.allclose(v, (1 - 0.999 ** t) * g * g, rtol=1e-12)
