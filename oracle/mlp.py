"""Oracle of the learned ROM error estimator (test infrastructure only).

The paper measures the reduced model's error against full-order solutions and
suggests replacing that by a cheaper estimate (Sec. 5).  The learned estimator
is a small fully connected network, 5 -> 64 -> 64 -> 1 with tanh hidden units,
trained by mean-squared error with Adam (Kingma & Ba 2015) on samples the
method computes itself: features (frequency, distances to the three nearest
expansion points, log10 of the residual estimate) and the log10 of the true
relative output error of the ROM at that frequency.

Plain FP64 numpy, written from the definitions.  `half_weights` rounds the
weight matrices to FP16, the storage format of the GPU network, so forward and
backward passes can be compared on the same weights.

Only tests/, __graft_entry__.smoke() and bench.py may import this module.
"""
from typing import Dict, List, Tuple

import numpy as np

LAYERS = (5, 64, 64, 1)
NAMES = ("W1", "b1", "W2", "b2", "W3", "b3")
SHAPES = {"W1": (64, 5), "b1": (64,), "W2": (64, 64), "b2": (64,), "W3": (1, 64), "b3": (1,)}
N_PARAMS = sum(int(np.prod(s)) for s in SHAPES.values())


def features(cand_hz, shifts_hz, est, lo: float, hi: float) -> np.ndarray:
    """Estimator inputs per candidate frequency (one row of 5): the position in the band
    (f - lo) / (hi - lo); the distances to the three nearest expansion points over the band
    width, capped at 1 (1 where there are fewer points); log10 of the residual estimate
    (floored at 1e-16) over 4."""
    cand = np.asarray(cand_hz, dtype=float)
    sh = np.asarray(shifts_hz, dtype=float)
    span = hi - lo if hi > lo else 1.0
    X = np.ones((cand.size, 5))
    X[:, 0] = (cand - lo) / span
    for i, f in enumerate(cand):
        d = np.sort(np.abs(f - sh) / span)[:3]
        X[i, 1:1 + d.size] = np.minimum(d, 1.0)
    X[:, 4] = np.log10(np.maximum(np.asarray(est, dtype=float), 1e-16)) / 4.0
    return X


def unflatten(flat: np.ndarray) -> Dict[str, np.ndarray]:
    """Parameters from the flat vector [W1 (row-major), b1, W2, b2, W3, b3]."""
    out, o = {}, 0
    for k in NAMES:
        n = int(np.prod(SHAPES[k]))
        out[k] = np.asarray(flat[o:o + n], dtype=np.float64).reshape(SHAPES[k]).copy()
        o += n
    return out


def flatten(p: Dict[str, np.ndarray]) -> np.ndarray:
    return np.concatenate([np.asarray(p[k], dtype=np.float64).ravel() for k in NAMES])


def half_weights(p: Dict[str, np.ndarray]) -> Dict[str, np.ndarray]:
    """Weight matrices rounded to FP16 (biases stay)."""
    q = {k: v.copy() for k, v in p.items()}
    for k in ("W1", "W2", "W3"):
        q[k] = p[k].astype(np.float16).astype(np.float64)
    return q


def forward(p, X: np.ndarray) -> Tuple[np.ndarray, tuple]:
    """y = W3 tanh(W2 tanh(W1 x + b1) + b2) + b3 for every row x of X (N x 5)."""
    h1 = np.tanh(X @ p["W1"].T + p["b1"])
    h2 = np.tanh(h1 @ p["W2"].T + p["b2"])
    y = (h2 @ p["W3"].T + p["b3"])[:, 0]
    return y, (X, h1, h2)


def mse(y: np.ndarray, t: np.ndarray) -> float:
    return float(np.mean((y - t) ** 2))


def backward(p, cache, y: np.ndarray, t: np.ndarray) -> Dict[str, np.ndarray]:
    """Gradient of mean((y - t)^2) with respect to every parameter (chain rule)."""
    X, h1, h2 = cache
    n = X.shape[0]
    dy = 2.0 * (y - t) / n                       # dL/dy
    g = {"W3": dy[None, :] @ h2, "b3": np.array([dy.sum()])}
    dz2 = (dy[:, None] @ p["W3"]) * (1.0 - h2 ** 2)
    g["W2"] = dz2.T @ h1
    g["b2"] = dz2.sum(axis=0)
    dz1 = (dz2 @ p["W2"]) * (1.0 - h1 ** 2)
    g["W1"] = dz1.T @ X
    g["b1"] = dz1.sum(axis=0)
    return g


def adam_step(p, g, m, v, step: int, lr: float, beta1: float = 0.9, beta2: float = 0.999,
              eps: float = 1e-8) -> None:
    """One Adam update in place (bias-corrected moments; step counts from 1)."""
    for k in NAMES:
        m[k] = beta1 * m[k] + (1.0 - beta1) * g[k]
        v[k] = beta2 * v[k] + (1.0 - beta2) * g[k] ** 2
        mh = m[k] / (1.0 - beta1 ** step)
        vh = v[k] / (1.0 - beta2 ** step)
        p[k] = p[k] - lr * mh / (np.sqrt(vh) + eps)


def train(p0, X: np.ndarray, T: np.ndarray, order: np.ndarray, lr: float = 1e-3,
          fp16: bool = True) -> Tuple[Dict[str, np.ndarray], List[float]]:
    """Mini-batch Adam: step s uses the rows order[s] (steps x batch).  With fp16 the
    forward and backward passes use FP16-rounded weights; the update is applied to the
    full-precision master weights."""
    p = {k: v.copy() for k, v in p0.items()}
    m = {k: np.zeros_like(v) for k, v in p.items()}
    v = {k: np.zeros_like(x) for k, x in p.items()}
    losses = []
    for s in range(order.shape[0]):
        idx = order[s]
        q = half_weights(p) if fp16 else p
        y, cache = forward(q, X[idx])
        losses.append(mse(y, T[idx]))
        adam_step(p, backward(q, cache, y, T[idx]), m, v, s + 1, lr)
    return p, losses
