"""Float64 CPU reference of the scheduler's cost model, for gradient checks.

TEST INFRASTRUCTURE ONLY (imported by tests/ alone).  The model is the
two-hidden-layer perceptron the scheduler uses: 8 inputs -> 64 -> 64 -> 1
with ReLU, trained by mean squared error.  Parameters are one flat vector
in the order W1 (64x8, row-major), b1 (64), W2 (64x64), b2 (64), W3 (64),
b3 (1).  Everything here is plain numpy in float64; gradients are written
out by the chain rule and pinned against central finite differences in the
tests.
"""
from __future__ import annotations

import numpy as np

N_IN, N_H = 8, 64
SIZES = [("W1", (N_H, N_IN)), ("b1", (N_H,)), ("W2", (N_H, N_H)), ("b2", (N_H,)), ("W3", (N_H,)), ("b3", (1,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SIZES)


def unpack(theta):
    out, o = {}, 0
    for name, shape in SIZES:
        n = int(np.prod(shape))
        out[name] = np.asarray(theta[o:o + n], np.float64).reshape(shape)
        o += n
    return out


def pack(p):
    return np.concatenate([np.asarray(p[name], np.float64).ravel() for name, _ in SIZES])


def forward(theta, X):
    p = unpack(theta)
    z1 = X @ p["W1"].T + p["b1"]
    h1 = np.maximum(z1, 0)
    z2 = h1 @ p["W2"].T + p["b2"]
    h2 = np.maximum(z2, 0)
    y = h2 @ p["W3"] + p["b3"][0]
    return y, (X, z1, h1, z2, h2)


def loss(theta, X, t):
    y, _ = forward(theta, X)
    return float(np.mean((y - t) ** 2))


def loss_grad(theta, X, t):
    """Mean squared error and its gradient (same flat layout as theta)."""
    p = unpack(theta)
    y, (X, z1, h1, z2, h2) = forward(theta, X)
    n = X.shape[0]
    dy = 2.0 * (y - t) / n                      # dL/dy
    g = {}
    g["W3"] = h2.T @ dy
    g["b3"] = np.array([dy.sum()])
    dz2 = np.outer(dy, p["W3"]) * (z2 > 0)
    g["W2"] = dz2.T @ h1
    g["b2"] = dz2.sum(axis=0)
    dz1 = (dz2 @ p["W2"]) * (z1 > 0)
    g["W1"] = dz1.T @ X
    g["b1"] = dz1.sum(axis=0)
    return float(np.mean((y - t) ** 2)), pack(g)


def finite_diff(theta, X, t, idx, eps=1e-6):
    """Central differences of the loss for the parameters at positions idx."""
    out = []
    for i in idx:
        a = theta.copy()
        b = theta.copy()
        a[i] += eps
        b[i] -= eps
        out.append((loss(a, X, t) - loss(b, X, t)) / (2 * eps))
    return np.array(out)
