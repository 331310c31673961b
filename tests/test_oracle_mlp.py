"""Pins for the oracle of the learned error estimator: the backward pass against
central finite differences, Adam's first step against its closed form, the forward
pass on weights with a closed-form output, and training on a smooth target."""
import numpy as np
import pytest

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


def test_features_pins_and_library_host_code():
    """Estimator inputs: a candidate on an expansion point has distance 0 to it; missing
    points read as distance 1; the band ends map to 0 and 1; the residual estimate enters
    as log10(est)/4.  The library's host routine (rom_features, C++) gives the same values
    in FP32."""
    cand = np.array([10.0, 12.5, 20.0, 30.0])
    sh = [12.5, 28.0]
    est = np.array([1e-4, 1e-20, 1.0, 3e-2])
    X = mlp.features(cand, sh, est, 10.0, 30.0)
    assert X.shape == (4, 5)
    assert X[0, 0] == 0.0 and X[3, 0] == 1.0
    assert X[1, 1] == 0.0 and X[1, 2] == pytest.approx(15.5 / 20.0) and X[1, 3] == 1.0
    assert X[0, 1] == pytest.approx(2.5 / 20.0) and X[0, 2] == pytest.approx(18.0 / 20.0)
    assert X[0, 4] == pytest.approx(-1.0) and X[1, 4] == pytest.approx(-4.0) and X[2, 4] == 0.0
    from paper_2310_04734_gb300 import api
    rng = np.random.default_rng(5)
    cand = np.sort(rng.uniform(1.0, 800.0, 200))
    sh = rng.uniform(1.0, 800.0, 7)
    est = 10.0 ** rng.uniform(-12, 1, 200)
    got = api.rom_features(cand, sh, est, cand[0], cand[-1])
    ref = mlp.features(cand, sh, est, cand[0], cand[-1])
    assert np.allclose(got, ref, rtol=2e-7, atol=2e-7)
    one = api.rom_features(cand[:5], sh[:1], est[:5], cand[0], cand[-1])
    assert np.all(one[:, 2:4] == 1.0)
