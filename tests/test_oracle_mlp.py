"""Pins for the oracle of the learned error estimator: the backward pass against
central finite differences, Adam's first step against its closed form, the forward
pass on weights with a closed-form output, and training on a smooth target."""
import numpy as np

import workloads as W
from oracle import mlp


def _data(n=64, seed=3):
    rng = np.random.default_rng(seed)
    X = rng.uniform(-1, 1, size=(n, 5))
    T = np.sin(2 * X[:, 0]) + 0.5 * X[:, 1] * X[:, 2] - 0.3 * X[:, 4]
    return X, T


def test_backward_matches_central_differences():
    p = mlp.unflatten(W.mlp_init())
    rng = np.random.default_rng(1)
    for k in mlp.NAMES:   # non-zero biases so every term of the chain rule is exercised
        p[k] = p[k] + 0.1 * rng.standard_normal(p[k].shape)
    X, T = _data()
    y, cache = mlp.forward(p, X)
    g = mlp.backward(p, cache, y, T)
    h = 1e-6
    for k in mlp.NAMES:
        num = np.zeros_like(p[k])
        it = np.nditer(p[k], flags=["multi_index"])
        for _ in it:
            i = it.multi_index
            q = {kk: vv.copy() for kk, vv in p.items()}
            q[k][i] += h
            lp = mlp.mse(mlp.forward(q, X)[0], T)
            q[k][i] -= 2 * h
            lm = mlp.mse(mlp.forward(q, X)[0], T)
            num[i] = (lp - lm) / (2 * h)
        assert np.abs(g[k] - num).max() <= 1e-6 * max(np.abs(num).max(), 1e-3), k


def test_forward_closed_form():
    # W1 = W2 = 0: y = W3 tanh(b2) + b3 for every input
    p = {k: np.zeros(s) for k, s in mlp.SHAPES.items()}
    p["b2"][:] = np.linspace(-1, 1, 64)
    p["W3"][0, :] = np.arange(64) / 64.0
    p["b3"][0] = 0.25
    X, _ = _data(5)
    y, _ = mlp.forward(p, X)
    assert np.allclose(y, (np.arange(64) / 64.0) @ np.tanh(np.linspace(-1, 1, 64)) + 0.25, rtol=0, atol=1e-15)


def test_adam_first_step_closed_form():
    # after one step the bias-corrected moments are g and g^2: update = -lr g / (|g| + eps)
    p = {k: np.ones(s) for k, s in mlp.SHAPES.items()}
    g = {k: np.full(s, -0.3) for k, s in mlp.SHAPES.items()}
    m = {k: np.zeros(s) for k, s in mlp.SHAPES.items()}
    v = {k: np.zeros(s) for k, s in mlp.SHAPES.items()}
    mlp.adam_step(p, g, m, v, 1, lr=1e-3)
    for k in mlp.NAMES:
        assert np.allclose(p[k], 1.0 + 1e-3 * 0.3 / (0.3 + 1e-8), rtol=0, atol=1e-15)


def test_training_fits_a_smooth_target():
    X, T = _data(n=2048, seed=5)
    p0 = mlp.unflatten(W.mlp_init())
    order = W.mlp_order(len(X), 600, 128)
    p, losses = mlp.train(p0, X, T, order, lr=3e-3)
    assert np.mean(losses[-50:]) < 0.1 * np.mean(losses[:10])
    assert mlp.mse(mlp.forward(p, X)[0], T) < 0.02


def test_half_weights_round_only_the_matrices():
    p = mlp.unflatten(W.mlp_init())
    q = mlp.half_weights(p)
    assert np.array_equal(q["b1"], p["b1"])
    assert np.abs(q["W2"] - p["W2"]).max() <= np.abs(p["W2"]).max() * 2.0 ** -11
    assert mlp.N_PARAMS == 64 * 5 + 64 + 64 * 64 + 64 + 64 + 1
