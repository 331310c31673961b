"""Design study with the learned error estimator (the reduced-order sweep of many
model variants; the paper's Sec. 5 outlook of a cheaper error estimate).

Only calls into the C-ABI: full-order sweeps, greedy ROMs, reduced sweeps, output
errors, estimator features, training and inference all run in the library's
kernels; this module sequences them and moves small host arrays.

Samples: for a variant, the greedy ROM after r = 1..rounds expansion points (the
greedy is deterministic, so the r-point ROM is the prefix of a longer run); at
every candidate frequency the features (rom_features) and the target
log10(relative output error vs the full-order sweep) / 4.
"""
from dataclasses import dataclass
from typing import List, Sequence

import numpy as np

from . import api


@dataclass
class VariantData:
    X: np.ndarray       # samples x 5 features (float32)
    T: np.ndarray       # samples: log10(true relative output error) / 4
    rounds: int
    cand: np.ndarray


def _setup(w):
    import torch
    model = api.fsi_assemble(w.model)
    F = api.dense_loads(w.model, w.loads, w.n_rhs)
    rcv = torch.tensor(api.receiver_dofs(w.model, w.receivers), device="cuda")
    return model, F, rcv


def full_order(w, model, F, rcv, batch: int = 32):
    """Receiver pressures of the full-order sweep (FP32 factor + FP64 GMRES to 1e-10)."""
    r = api.frf_sweep_full(model, w.freqs_hz, F, rcv, precision="fp32_ir", batch=batch, max_refine=60, tol=1e-10,
                           allow_noconv=True)
    return r.p


def variant_samples(w, rounds: int, q: int, kmax: int) -> VariantData:
    model, F, rcv = _setup(w)
    cand = np.asarray(w.freqs_hz, dtype=np.float64)
    pfull = full_order(w, model, F, rcv)
    Xs, Ts = [], []
    for r in range(1, rounds + 1):
        g = api.rom_greedy(model, F, rcv, cand, q=q, kmax=kmax, max_shifts=r, tol=0.0)
        p, _ = api.rom_sweep(g.rom, cand, batch=128)
        err = api.rom_output_error(pfull, p).cpu().numpy()
        Xs.append(api.rom_features(cand, g.shifts_hz, g.est, cand[0], cand[-1]))
        Ts.append((np.log10(np.maximum(err, 1e-16)) / 4.0).astype(np.float32))
    return VariantData(X=np.concatenate(Xs), T=np.concatenate(Ts), rounds=rounds, cand=cand)


def train_estimator(data: Sequence[VariantData], init_params, order, lr: float = 1e-3):
    """Adam on the pooled samples; order: steps x batch rows of the pooled set."""
    X = np.concatenate([d.X for d in data])
    T = np.concatenate([d.T for d in data])
    st = api.mlp_state(init_params)
    losses = api.mlp_train(st, X, T, order, lr=lr)
    return st, losses.cpu().numpy()


def greedy_error(w, rounds: int, q: int, kmax: int, mlp_params=None):
    """Largest true relative output error over the candidates after `rounds` points,
    with the residual-driven or the estimator-driven greedy."""
    model, F, rcv = _setup(w)
    cand = np.asarray(w.freqs_hz, dtype=np.float64)
    pfull = full_order(w, model, F, rcv)
    g = api.rom_greedy(model, F, rcv, cand, q=q, kmax=kmax, max_shifts=rounds, tol=0.0, mlp_params=mlp_params)
    p, _ = api.rom_sweep(g.rom, cand, batch=128)
    err = api.rom_output_error(pfull, p).cpu().numpy()
    return float(err.max()), g.shifts_hz


def rmse(a, b) -> float:
    return float(np.sqrt(np.mean((np.asarray(a, dtype=np.float64) - np.asarray(b, dtype=np.float64)) ** 2)))


def linear_baseline(train: List[VariantData]):
    """Least-squares fit T ~ a * x4 + c (the residual estimate alone as error predictor)."""
    x = np.concatenate([d.X[:, 4] for d in train]).astype(np.float64)
    t = np.concatenate([d.T for d in train]).astype(np.float64)
    A = np.stack([x, np.ones_like(x)], axis=1)
    coef, *_ = np.linalg.lstsq(A, t, rcond=None)
    return coef


def variant_rom(w, q: int, kmax: int, max_shifts: int, tol: float, mlp_params=None):
    """Greedy ROM of one variant over its frequency grid (residual- or estimator-driven)."""
    model, F, rcv = _setup(w)
    cand = np.asarray(w.freqs_hz, dtype=np.float64)
    g = api.rom_greedy(model, F, rcv, cand, q=q, kmax=kmax, max_shifts=max_shifts, tol=tol, mlp_params=mlp_params)
    return g, (model, F, rcv)


def check_variant(w, handles, p_rom, check_idx):
    """Full-order solutions at the check frequencies and the ROM's SPL error there (dB);
    frequencies above 0.1 dB are the ones to re-solve at full order."""
    model, F, rcv = handles
    f = np.asarray(w.freqs_hz, dtype=np.float64)[check_idx]
    r = api.frf_sweep_full(model, f, F, rcv, precision="fp32_ir", batch=len(f), max_refine=60, tol=1e-10,
                           allow_noconv=True)
    pf = r.p.cpu().numpy()
    pr = p_rom[check_idx].cpu().numpy()
    db = np.abs(20.0 * np.log10(np.abs(pr) / np.abs(pf))).max(axis=(1, 2))
    return db, pf
