"""Pins for the float64 reference of the scheduler's cost model."""
import numpy as np

from oracle import mlp


def _data(seed, n=40):
    rng = np.random.default_rng(seed)
    theta = rng.normal(0, 0.3, mlp.N_PARAMS)
    X = rng.normal(0, 1, (n, mlp.N_IN))
    t = rng.normal(0, 1, n)
    return theta, X, t


def test_gradient_matches_finite_differences():
    theta, X, t = _data(1)
    _, g = mlp.loss_grad(theta, X, t)
    rng = np.random.default_rng(2)
    idx = np.concatenate([rng.choice(mlp.N_PARAMS, 60, replace=False), [mlp.N_PARAMS - 1, 0, 600]])
    fd = mlp.finite_diff(theta, X, t, idx)
    assert np.allclose(g[idx], fd, rtol=1e-5, atol=1e-8)


def test_zero_hidden_weights_give_bias_only():
    theta, X, t = _data(3)
    p = mlp.unpack(theta)
    p["W3"][:] = 0
    th = mlp.pack(p)
    y, _ = mlp.forward(th, X)
    assert np.allclose(y, p["b3"][0])
    loss, g = mlp.loss_grad(th, X, t)
    # d/db3 of mean (b3 - t)^2 = 2 * mean(b3 - t)
    assert np.isclose(g[-1], 2 * np.mean(p["b3"][0] - t))
    assert np.isclose(loss, np.mean((p["b3"][0] - t) ** 2))


def test_relu_inactive_units_get_no_gradient():
    theta, X, t = _data(4)
    p = mlp.unpack(theta)
    p["b1"][:5] = -1e6            # units 0..4 of layer 1 never fire
    th = mlp.pack(p)
    _, g = mlp.loss_grad(th, X, t)
    G = mlp.unpack(g)
    assert np.all(G["W1"][:5] == 0) and np.all(G["b1"][:5] == 0)
    assert np.all(G["W2"][:, :5] == 0)
