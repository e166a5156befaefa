"""FP64 reference of the learned stopping predictor -- TEST INFRASTRUCTURE.

A multilayer perceptron 64 -> 256 -> 256 -> 2 with exact GELU
(gelu(z) = z * Phi(z), Phi the standard normal CDF) after the two hidden
layers and a linear output, trained on the mean squared error
L = (1 / (2 B)) * sum_b ||y_b - target_b||^2 with Adam (Kingma and Ba, 2015:
m <- b1 m + (1 - b1) g, v <- b2 v + (1 - b2) g^2, p <- p - lr * mhat / (sqrt(vhat) + eps),
mhat = m / (1 - b1^t), vhat = v / (1 - b2^t)).  The paper has no learned part;
this follows the architecture the build specifies.

Parameters are kept as one flat vector in the order W1 (256x64, row-major),
b1 (256), W2 (256x256), b2 (256), W3 (2x256), b3 (2), the layout the CUDA
kernels use.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf

SIZES = (64, 256, 256, 2)


def shapes():
    d0, d1, d2, d3 = SIZES
    return [("W1", (d1, d0)), ("b1", (d1,)), ("W2", (d2, d1)), ("b2", (d2,)), ("W3", (d3, d2)), ("b3", (d3,))]


def n_params() -> int:
    return sum(int(np.prod(s)) for _, s in shapes())


def unpack(theta):
    out, o = {}, 0
    for name, s in shapes():
        k = int(np.prod(s))
        out[name] = theta[o:o + k].reshape(s)
        o += k
    return out


def pack(d):
    return np.concatenate([np.asarray(d[name], dtype=np.float64).reshape(-1) for name, _ in shapes()])


def init_params(seed: int) -> np.ndarray:
    """Kaiming-uniform weights (bound sqrt(6 / fan_in)) and zero biases, seeded."""
    rng = np.random.default_rng(seed)
    d = {}
    for name, s in shapes():
        if name.startswith("W"):
            bound = math.sqrt(6.0 / s[1])
            d[name] = rng.uniform(-bound, bound, size=s)
        else:
            d[name] = np.zeros(s)
    return pack(d)


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / math.sqrt(2.0)))


def gelu_grad(z):
    return 0.5 * (1.0 + erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def forward(theta, X):
    p = unpack(theta)
    Z1 = X @ p["W1"].T + p["b1"]
    H1 = gelu(Z1)
    Z2 = H1 @ p["W2"].T + p["b2"]
    H2 = gelu(Z2)
    Y = H2 @ p["W3"].T + p["b3"]
    return Y, (X, Z1, H1, Z2, H2)


def loss(theta, X, T):
    Y, _ = forward(theta, X)
    return 0.5 * float(np.sum((Y - T) ** 2)) / X.shape[0]


def gradient(theta, X, T):
    """dL/dtheta by the chain rule, in the flat parameter order."""
    p = unpack(theta)
    Y, (X, Z1, H1, Z2, H2) = forward(theta, X)
    B = X.shape[0]
    dY = (Y - T) / B
    g = {"W3": dY.T @ H2, "b3": dY.sum(axis=0)}
    dZ2 = (dY @ p["W3"]) * gelu_grad(Z2)
    g["W2"] = dZ2.T @ H1
    g["b2"] = dZ2.sum(axis=0)
    dZ1 = (dZ2 @ p["W2"]) * gelu_grad(Z1)
    g["W1"] = dZ1.T @ X
    g["b1"] = dZ1.sum(axis=0)
    return pack(g)


def adam_step(theta, m, v, grad, step, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update; `step` counts from 1.  Returns (theta, m, v)."""
    m = b1 * m + (1.0 - b1) * grad
    v = b2 * v + (1.0 - b2) * grad * grad
    mhat = m / (1.0 - b1 ** step)
    vhat = v / (1.0 - b2 ** step)
    return theta - lr * mhat / (np.sqrt(vhat) + eps), m, v
