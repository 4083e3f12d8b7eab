"""FP64 CPU oracle of the learned coarse-grid correction network.

TEST INFRASTRUCTURE ONLY (tests, smoke check, CPU baseline).  Plain numpy,
written from the definition, sharing no code with the CUDA kernels.

Network (a per-cell multilayer perceptron): 76 inputs -> Linear(64) -> GELU ->
Linear(64) -> GELU -> Linear(4); GELU(x) = x Phi(x) with the exact normal CDF.
Parameters are laid out in one flat vector
    [W1 (64x76, row-major out x in), b1 (64), W2 (64x64), b2 (64), W3 (4x64), b3 (4)]
= 9,348 values.  Loss: mean squared error over samples and outputs.  Adam with
bias correction (Kingma and Ba, "Adam: a method for stochastic optimization",
ICLR 2015).
"""
from __future__ import annotations

import math

import numpy as np

SIZES = [(64, 76), (64, 64), (4, 64)]
N_PARAMS = sum(o * i + o for o, i in SIZES)


def unpack(theta):
    out, k = [], 0
    for o, i in SIZES:
        W = theta[k:k + o * i].reshape(o, i)
        k += o * i
        b = theta[k:k + o]
        k += o
        out.append((W, b))
    return out


def gelu(x):
    return 0.5 * x * (1.0 + np.vectorize(math.erf)(x / math.sqrt(2.0)))


def gelu_grad(x):
    cdf = 0.5 * (1.0 + np.vectorize(math.erf)(x / math.sqrt(2.0)))
    pdf = np.exp(-0.5 * x * x) / math.sqrt(2.0 * math.pi)
    return cdf + x * pdf


def forward(theta, X):
    """Returns the prediction and the cached pre-activations."""
    (W1, b1), (W2, b2), (W3, b3) = unpack(theta)
    Z1 = X @ W1.T + b1
    A1 = gelu(Z1)
    Z2 = A1 @ W2.T + b2
    A2 = gelu(Z2)
    Y = A2 @ W3.T + b3
    return Y, (X, Z1, A1, Z2, A2)


def loss(theta, X, Y):
    P, _ = forward(theta, X)
    return float(np.mean((P - Y) ** 2))


def grad(theta, X, Y):
    """Analytic gradient of the mean squared error (chain rule, layer by layer)."""
    (W1, b1), (W2, b2), (W3, b3) = unpack(theta)
    P, (X, Z1, A1, Z2, A2) = forward(theta, X)
    dP = 2.0 * (P - Y) / P.size
    gW3 = dP.T @ A2
    gb3 = dP.sum(0)
    dA2 = dP @ W3
    dZ2 = dA2 * gelu_grad(Z2)
    gW2 = dZ2.T @ A1
    gb2 = dZ2.sum(0)
    dA1 = dZ2 @ W2
    dZ1 = dA1 * gelu_grad(Z1)
    gW1 = dZ1.T @ X
    gb1 = dZ1.sum(0)
    return np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3])


def adam_step(theta, g, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (t counts from 1); returns new (theta, m, v)."""
    m = beta1 * m + (1 - beta1) * g
    v = beta2 * v + (1 - beta2) * g * g
    mh = m / (1 - beta1 ** t)
    vh = v / (1 - beta2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


def to_bf16(x):
    """Round to the nearest bfloat16 (ties to even) and return as float64."""
    a = np.ascontiguousarray(x, np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    rounded = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return rounded.astype(np.uint32).view(np.float32).astype(np.float64)


def init_params(seed=0):
    """Seeded He-style initialisation (the learned part's input generator)."""
    rng = np.random.default_rng(seed)
    parts = []
    for o, i in SIZES:
        parts.append(rng.standard_normal(o * i) * math.sqrt(2.0 / i))
        parts.append(np.zeros(o))
    return np.concatenate(parts)
