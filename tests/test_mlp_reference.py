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


def test_forward_hand_evaluated():
    """Forward pass against values worked out by hand, with both ReLU layers
    deciding the result: hidden unit 1 of layer 1 is cut for x0 > 0 and unit
    0 for x0 < 0; unit 0 of layer 2 is cut for the third sample."""
    p = {name: np.zeros(shape) for name, shape in mlp.SIZES}
    p["W1"][0, 0], p["W1"][1, 0] = 1.0, -1.0      # h1_0 = relu(x0), h1_1 = relu(-x0)
    p["b1"][2] = 0.5                               # h1_2 = 0.5
    p["W2"][0, 0], p["W2"][0, 1], p["b2"][0] = 2.0, 3.0, -1.0   # z2_0 = 2 h1_0 + 3 h1_1 - 1
    p["W2"][1, 2] = 1.0                            # z2_1 = h1_2
    p["W3"][0], p["W3"][1], p["b3"][0] = 1.0, 4.0, 0.25         # y = h2_0 + 4 h2_1 + 1/4
    X = np.zeros((3, mlp.N_IN))
    X[:, 0] = [2.0, -1.0, 0.1]
    X[:, 5] = [7.0, -3.0, 1.0]                     # a feature no weight reads
    # x0 = 2:   h1 = (2, 0, .5),  z2_0 = 3,     y = 3 + 2 + .25
    # x0 = -1:  h1 = (0, 1, .5),  z2_0 = 2,     y = 2 + 2 + .25
    # x0 = .1:  h1 = (.1, 0, .5), z2_0 = -0.8,  y = 0 + 2 + .25
    y, (_, z1, h1, z2, h2) = mlp.forward(mlp.pack(p), X)
    assert np.allclose(y, [5.25, 4.25, 2.25], rtol=0, atol=1e-12)
    assert np.allclose(z2[:, 0], [3.0, 2.0, -0.8]) and np.allclose(h2[:, 0], [3.0, 2.0, 0.0])
    assert np.allclose(h1[:, :3], [[2, 0, .5], [0, 1, .5], [.1, 0, .5]])
    # the loss at these outputs against targets (5, 5, 2): mean of .0625, .5625, .0625
    assert np.isclose(mlp.loss(mlp.pack(p), X, np.array([5.0, 5.0, 2.0])), (0.0625 + 0.5625 + 0.0625) / 3)
