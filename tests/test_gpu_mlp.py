"""The estimator's GPU training kernel against the oracle (same FP16-rounded weights,
same seeded initialisation and batch order): loss and gradient of a full batch,
the parameters after a few Adam steps, and a full training run's final loss; the
inference kernel against the oracle's forward pass."""
import numpy as np
import pytest

import workloads as W
from gpu_util import need_cuda
from oracle import mlp

pytestmark = pytest.mark.gpu


def _data(n, seed):
    rng = np.random.default_rng(seed)
    X = rng.uniform(-1, 1, size=(n, 5))
    T = np.sin(2 * X[:, 0]) + 0.5 * X[:, 1] * X[:, 2] - 0.3 * X[:, 4]
    return X, T


def test_gradient_matches_oracle_backward():
    need_cuda()
    from paper_2310_04734_gb300 import api
    X, T = _data(256, 7)
    p0 = W.mlp_init()
    p0 = p0 + 0.05 * np.random.default_rng(2).standard_normal(p0.size)   # non-zero biases
    st = api.mlp_state(p0)
    order = np.arange(256, dtype=np.int32)[None, :]
    losses, g = api.mlp_train(st, X, T, order, lr=0.0, want_grad=True)
    q = mlp.half_weights(mlp.unflatten(p0.astype(np.float32).astype(np.float64)))
    y, cache = mlp.forward(q, X.astype(np.float32).astype(np.float64))
    gref = mlp.flatten(mlp.backward(q, cache, y, T.astype(np.float32).astype(np.float64)))
    gg = g.cpu().numpy().astype(np.float64)
    assert abs(losses.item() - mlp.mse(y, T)) <= 1e-4 * mlp.mse(y, T)
    for k, (a, b) in zip(mlp.NAMES, np.split(np.stack([gg, gref]), np.cumsum(
            [int(np.prod(mlp.SHAPES[k])) for k in mlp.NAMES])[:-1], axis=1)):
        assert np.abs(a - b).max() <= 1e-3 * np.abs(b).max(), k


def test_adam_steps_and_training_match_oracle():
    need_cuda()
    from paper_2310_04734_gb300 import api
    X, T = _data(4096, 9)
    p0 = W.mlp_init()
    order = W.mlp_order(len(X), 400, 128)
    st = api.mlp_state(p0)
    api.mlp_train(st, X, T, order[:5], lr=3e-3)
    pref, _ = mlp.train(mlp.unflatten(p0.astype(np.float32).astype(np.float64)), X.astype(np.float32),
                        T.astype(np.float32), order[:5], lr=3e-3)
    got = st.params.cpu().numpy().astype(np.float64)
    ref = mlp.flatten(pref)
    d = np.abs(got - ref)
    # Adam normalises each update to ~lr, so a parameter whose gradient is at the FP32
    # rounding level may step either way: bound those by the steps taken
    assert np.quantile(d, 0.999) <= 1e-3 * np.abs(ref).max() and d.max() <= 2 * 5 * 3e-3
    losses = api.mlp_train(st, X, T, order[5:], lr=3e-3).cpu().numpy()
    _, lref = mlp.train(mlp.unflatten(p0.astype(np.float32).astype(np.float64)), X.astype(np.float32),
                        T.astype(np.float32), order, lr=3e-3)
    print("final loss gpu %.5f oracle %.5f" % (losses[-20:].mean(), np.mean(lref[-20:])))
    assert abs(losses[-20:].mean() - np.mean(lref[-20:])) <= 0.05 * np.mean(lref[-20:]) + 1e-4
    assert losses[-20:].mean() < 0.1 * np.mean(lref[:5])


def test_predict_matches_oracle_forward():
    need_cuda()
    from paper_2310_04734_gb300 import api
    X, _ = _data(1000, 11)
    p0 = W.mlp_init() + 0.05 * np.random.default_rng(3).standard_normal(W.mlp_init().size)
    st = api.mlp_state(p0)
    y = api.mlp_predict(st.params, X).cpu().numpy()
    q = mlp.half_weights(mlp.unflatten(p0.astype(np.float32).astype(np.float64)))
    yref, _ = mlp.forward(q, X.astype(np.float32).astype(np.float64))
    assert np.abs(y - yref).max() <= 1e-4 * max(np.abs(yref).max(), 1.0)
