"""Oracle rational Arnoldi model order reduction (TEST INFRASTRUCTURE ONLY).

Follows the paper's Sec. 3.3 step by step:

* projection basis: union over expansion points w_j of the Krylov subspaces
  - second order (Eq. 9):  K(-Kt_j^-1 Dt_j, -Kt_j^-1 Mt_j; -Kt_j^-1 f_j) with
    Kt_j = A(w_j), Dt_j = 2 i w_j M + D, Mt_j = M, built with the SOAR
    recurrence of Bai and Su (2005), the paper's reference for Eq. 9;
  - first order (Eq. 10) when there is no damping matrix (structural damping
    enters as complex stiffness): K(-Kt_j^-1 M, -Kt_j^-1 f_j).
  The shifted matrix Kt_j is factored once per expansion point and reused
  for every moment of that point (Sec. 3.3, offline phase).
  Moments are load specific: one starting vector per load column.
* every new vector is orthonormalised against the basis by classical
  Gram-Schmidt applied twice (CGS2), and dropped when its norm after the two
  passes is below 1e-10 of its norm before them (deflation).
* Galerkin projection (text after Eq. 11): [.]_R = V^H [.] V for K, D, M,
  f_R = V^H f (the paper prints V^T f; for a complex V the Galerkin
  projection needs V^H), y_R = C_R x_R with C_R = C^T V.
* reduced sweep: dense GEPP of K_R + i w D_R - w^2 M_R at every frequency.
* error measure eps(w) = |y - y_R| / |y| and eps_max = max_w eps(w)
  (Sec. 3.3; the paper writes arg max, the value is what is tabulated).
* greedy choice of expansion points (Sec. 3.3): the next point is the
  candidate frequency with the largest estimated error; here the estimator
  is the relative residual of the scaled full-order system.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import List, Optional

import numpy as np

from . import fom

DEFLATION_TOL = 1e-10


def cgs2_append(V: np.ndarray, W: np.ndarray, tol: float = DEFLATION_TOL):
    """Append the columns of W to the orthonormal V, one at a time, by CGS2.

    Returns (V_new, accepted) where ``accepted`` are the orthonormalised new columns.
    """
    cols = [V[:, i] for i in range(V.shape[1])]
    new = []
    for w in np.asarray(W).T:
        w = w.astype(complex).copy()
        pre = np.linalg.norm(w)
        if pre == 0.0:
            continue
        for _ in range(2):
            if cols:
                Q = np.stack(cols, axis=1)
                h = Q.conj().T @ w
                w = w - Q @ h
        nw = np.linalg.norm(w)
        if nw <= tol * pre:
            continue
        q = w / nw
        cols.append(q)
        new.append(q)
    Vn = np.stack(cols, axis=1) if cols else np.zeros((V.shape[0], 0), dtype=complex)
    An = np.stack(new, axis=1) if new else np.zeros((V.shape[0], 0), dtype=complex)
    return Vn, An


def _first_order_moments(asm, lu, F, q):
    """Moments of Eq. 10 at one expansion point: v_0 = Kt^-1 f, v_m = Kt^-1 M v_{m-1}."""
    out = []
    v = lu.solve(F)
    out.append(v)
    for _ in range(1, q):
        v = lu.solve(asm.M @ v)
        out.append(v)
    return out


def _soar(asm, lu, omega_j, f, q):
    """SOAR (Bai and Su 2005) for the second-order Krylov space of Eq. 9.

    A = -Kt^-1 Dt, B = -Kt^-1 M, starting vector u = -Kt^-1 f.  Returns an
    orthonormal basis of span{r_0, ..., r_{q-1}} with r_1 = A r_0,
    r_m = A r_{m-1} + B r_{m-2}.

    Each step forms r = A q_j + B p_j and the companion s = q_j, orthogonalises
    r against the q's (the same coefficients update s against the p's) and
    normalises both by |r|.  Deflation (|r| at rounding level, r already in
    the span): Bai and Su continue with q_{j+1} = 0 and p_{j+1} = s, so the
    sequence can still reach new directions later; the process breaks down
    (stops) only when s also lies in the span of the p vectors of earlier
    deflations.  Zero q's are not part of the returned basis.
    """
    Dt = 2j * omega_j * asm.M + asm.D
    u = -lu.solve(f)
    nu = np.linalg.norm(u)
    Q = [u / nu]
    P = [np.zeros_like(u)]
    deflated = []          # indices j with q_j = 0
    for j in range(q - 1):
        r = -lu.solve(Dt @ Q[j] + asm.M @ P[j])
        s = Q[j].copy()
        for i in range(j + 1):
            t = np.vdot(Q[i], r)
            r = r - t * Q[i]
            s = s - t * P[i]
        t = np.linalg.norm(r)
        if t > DEFLATION_TOL * nu:
            Q.append(r / t)
            P.append(s / t)
            continue
        # deflation: breakdown if s is in span{p_i : q_i = 0} (for none: s = 0)
        ns = np.linalg.norm(s)
        if deflated:
            Pd = np.stack([P[i] for i in deflated], axis=1)
            coef, *_ = np.linalg.lstsq(Pd, s, rcond=None)
            rest = np.linalg.norm(s - Pd @ coef)
        else:
            rest = ns
        if rest <= DEFLATION_TOL * max(ns, 1.0):
            break
        Q.append(np.zeros_like(u))
        P.append(s)
        deflated.append(j + 1)
    keep = [Q[i] for i in range(len(Q)) if i not in deflated]
    return np.stack(keep, axis=1)


def has_damping_matrix(asm) -> bool:
    return asm.D.nnz > 0 and abs(asm.D).max() > 0.0


def build_basis(asm, shifts_hz, q: int, F: np.ndarray, kmax: int, V0=None):
    """Rational Arnoldi basis: union over the expansion points of Eq. 9 / Eq. 10 moments.

    For each expansion point the shifted matrix is factored once; every load
    column contributes q moments; each new vector is CGS2-orthonormalised
    against everything accepted so far.  Stops at kmax columns.
    """
    V = np.zeros((asm.n, 0), dtype=complex) if V0 is None else V0
    second = has_damping_matrix(asm)
    for fj in shifts_hz:
        om = 2.0 * np.pi * fj
        lu = fom.BlockBandedLU(asm, om)
        if second:
            for c in range(F.shape[1]):
                V, _ = cgs2_append(V, _soar(asm, lu, om, F[:, c], q))
        else:
            for blk in _first_order_moments(asm, lu, F, q):
                V, _ = cgs2_append(V, blk)
        if V.shape[1] >= kmax:
            V = V[:, :kmax]
            break
    return V


@dataclass
class ReducedModel:
    KR: np.ndarray
    DR: np.ndarray
    MR: np.ndarray
    fR: np.ndarray
    CR: np.ndarray

    @property
    def k(self) -> int:
        return self.KR.shape[0]


def project(asm, V: np.ndarray, F: np.ndarray, rcv_dofs) -> ReducedModel:
    """Galerkin projection [.]_R = V^H [.] V, f_R = V^H f, C_R = C^T V (Sec. 3.3)."""
    VH = V.conj().T
    return ReducedModel(KR=VH @ (asm.K @ V), DR=VH @ (asm.D @ V), MR=VH @ (asm.M @ V),
                        fR=VH @ F, CR=V[np.asarray(rcv_dofs)])


def reduced_sweep(rm: ReducedModel, freqs_hz):
    """y_R(w) = C_R (K_R + i w D_R - w^2 M_R)^-1 f_R at every frequency (Eq. 11)."""
    out = np.empty((len(freqs_hz), rm.CR.shape[0], rm.fR.shape[1]), dtype=complex)
    for i, f in enumerate(freqs_hz):
        om = 2.0 * np.pi * f
        AR = rm.KR + 1j * om * rm.DR - om ** 2 * rm.MR
        out[i] = rm.CR @ np.linalg.solve(AR, rm.fR)
    return out


def relative_error(y: np.ndarray, yR: np.ndarray) -> np.ndarray:
    """eps(w) = |y - y_R| / |y| elementwise (Sec. 3.3)."""
    return np.abs(y - yR) / np.abs(y)


def residual_estimate(asm, V, rm: ReducedModel, F, freqs_hz) -> np.ndarray:
    """Relative residual ||R (F - A(w) V x_R)|| / ||R F|| of the scaled system, per frequency."""
    out = np.empty(len(freqs_hz))
    for i, f in enumerate(freqs_hz):
        om = 2.0 * np.pi * f
        AR = rm.KR + 1j * om * rm.DR - om ** 2 * rm.MR
        xR = np.linalg.solve(AR, rm.fR)
        r_s, _ = fom.equilibrate(asm, om)
        res = r_s[:, None] * (F - asm.A(om) @ (V @ xR))
        out[i] = np.linalg.norm(res) / np.linalg.norm(r_s[:, None] * F)
    return out


def full_residual(asm, V, rm: ReducedModel, F, freqs_hz) -> np.ndarray:
    """Plain relative residual of the lifted reduced solution in the full model, per load
    column: ||f_c - A(w) V x_R,c||_2 / ||f_c||_2 with A(w) = K + i w D - w^2 M (Eq. 8) and
    x_R the reduced solution (Eq. 11).  Shape [len(freqs_hz)][n_columns]."""
    out = np.empty((len(freqs_hz), F.shape[1]))
    fn = np.linalg.norm(F, axis=0)
    for i, f in enumerate(freqs_hz):
        om = 2.0 * np.pi * f
        AR = rm.KR + 1j * om * rm.DR - om ** 2 * rm.MR
        x = V @ np.linalg.solve(AR, rm.fR)
        out[i] = np.linalg.norm(F - asm.A(om) @ x, axis=0) / fn
    return out


def greedy(asm, F, rcv_dofs, cand_hz, q: int, kmax: int, tol: float, max_shifts: int,
           initial_hz: Optional[List[float]] = None):
    """Greedy expansion points: add the candidate with the largest residual estimate.

    Ties go to the lowest frequency; candidates within one grid step of an
    existing point are skipped.  Stops when the largest estimate is <= tol,
    after max_shifts points, or at kmax columns.
    """
    cand_hz = np.asarray(cand_hz, dtype=float)
    step = np.min(np.diff(cand_hz)) if len(cand_hz) > 1 else 0.0
    shifts = list(initial_hz) if initial_hz else [float(cand_hz[len(cand_hz) // 2])]
    V = build_basis(asm, shifts, q, F, kmax)
    history = []
    while True:
        rm = project(asm, V, F, rcv_dofs)
        est = residual_estimate(asm, V, rm, F, cand_hz)
        history.append(float(est.max()))
        if est.max() <= tol or len(shifts) >= max_shifts or V.shape[1] >= kmax:
            break
        order = np.argsort(-est, kind="stable")
        nxt = None
        for i in order:
            if all(abs(cand_hz[i] - s) > step * 1.0001 for s in shifts):
                nxt = float(cand_hz[i])
                break
        if nxt is None:
            break
        shifts.append(nxt)
        V = build_basis(asm, [nxt], q, F, kmax, V0=V)
    return shifts, V, project(asm, V, F, rcv_dofs), history


def windows(asm, F, rcv_dofs, cand_hz, q: int, kmax: int, tol: float, max_shifts: int,
            max_windows: int, min_points: int, reuse: bool = True):
    """Local ROMs over frequency windows (Sec. 3.3: one fROM per window).

    The candidate band starts as one window.  A window whose greedy ends with its
    largest estimate above tol is bisected by candidate count (left half first), down
    to min_points candidates and at most max_windows windows in all.  Each window's
    greedy starts from the expansion points of the windows it was split from that lie
    in its band (in the order they were chosen; with reuse), else from the candidates
    nearest its quarter midpoints.
    """
    cand_hz = np.asarray(cand_hz, dtype=float)
    todo = [(0, len(cand_hz))]
    out = []
    split = []   # (i0, i1, shifts) of the windows that were bisected, outermost first
    while todo:
        i0, i1 = todo.pop(0)
        c = cand_hz[i0:i1]
        split = [a for a in split if a[0] <= i0 and i1 <= a[1]]
        init = []
        if reuse:
            for a in split:
                for sh in a[2]:
                    if c[0] <= sh <= c[-1] and sh not in init:
                        init.append(sh)
            init = init[:max_shifts]
        nreused = len(init)
        if not init:
            for qq in range(4):
                t = c[0] + (c[-1] - c[0]) * (qq + 0.5) / 4.0
                pick = float(c[int(np.argmin(np.abs(c - t)))])
                if pick not in init and len(init) < max_shifts:
                    init.append(pick)
        shifts, V, rm, hist = greedy(asm, F, rcv_dofs, c, q, kmax, tol, max_shifts, initial_hz=init)
        mx = hist[-1]
        if mx > tol and (i1 - i0) >= 2 * max(1, min_points) and len(out) + len(todo) + 2 <= max_windows:
            mid = i0 + (i1 - i0) // 2
            todo[0:0] = [(i0, mid), (mid, i1)]
            split.append((i0, i1, shifts))
            continue
        out.append(dict(lo=float(c[0]), hi=float(c[-1]), shifts=shifts, V=V, rm=rm, maxest=mx, reused=nreused))
    return out
