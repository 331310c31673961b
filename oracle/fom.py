"""Oracle full-order frequency response (TEST INFRASTRUCTURE ONLY).

The full-order model (paper Sec. 2, Eq. 1, and Sec. 3.3, Eq. 8) is solved at
each frequency as its plain definition x(w) = A(w)^-1 f, A(w) = K + i w D -
w^2 M, followed by y = C^T x at the receiver pressure DoFs (Eq. 8) and the
sound pressure level.  Two independent routes:

* ``solve_dense``: the dense matrix and LAPACK's GEPP (numpy.linalg.solve),
  for tiny meshes.
* ``BlockBandedLU``: a banded complex LU with partial pivoting across the
  stacked panel [A_kk; A_{k+1,k}] of the slab-ordered matrix (the structure a
  general band GEPP such as zgbtrf would exploit, written out block by block).
  Row swaps between slab k and k+1 create the usual fill of one extra block
  superdiagonal in U.

Both first apply an exact diagonal scaling (R A C) y = R f, x = C y.  The
coupled u-p matrix is unsymmetric: its fluid rows carry -w^2 rho C^T where
the shell rows carry -C.  Dividing the fluid rows by rho w^2 (and negating
the fluid unknowns, which does not change magnitudes) makes it complex
symmetric, the algebraic form of acoustic-structural reciprocity; a symmetric
Jacobi scaling by |K_ii|^-1/2 then balances pressure and displacement
unknowns.  With the generic row/column max equilibration instead, the
condition number of the config-1 model is about 6e10 (it is about 1e6 with
this scaling), and two backward-stable solvers then disagree at 1e-8.
SPL uses the RMS convention L = 20 log10(|p| / (sqrt(2) * 20 uPa)).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as la
import scipy.sparse as sp

P_REF = 2e-5


def equilibrate(asm, omega: float):
    """Row and column scalings (r, c) of the reciprocity-symmetrised, Jacobi-scaled system.

    Fluid DoF i: r_i = 1 / (w sqrt(rho |K_ii|)), c_i = w sqrt(rho / |K_ii|);
    shell DoF i: r_i = c_i = 1 / sqrt(|K_ii|).
    """
    kd = np.abs(asm.K.diagonal())
    fl = asm.is_fluid
    rho = asm.spec.rho
    r = np.where(fl, 1.0 / (omega * np.sqrt(rho * kd)), 1.0 / np.sqrt(kd))
    c = np.where(fl, omega * np.sqrt(rho / kd), 1.0 / np.sqrt(kd))
    return r, c


def solve_dense(asm, omega: float, F: np.ndarray) -> np.ndarray:
    """x = A(w)^-1 F through the dense scaled matrix and LAPACK GEPP."""
    A = asm.A(omega)
    r, c = equilibrate(asm, omega)
    As = (sp.diags(r) @ A @ sp.diags(c)).toarray()
    y = np.linalg.solve(As, r[:, None] * F)
    return c[:, None] * y


class BlockBandedLU:
    """Banded complex GEPP of a block-tridiagonal matrix with nz blocks of size b.

    Pivoting searches the stacked 2b x b panel [A_kk; A_{k+1,k}], so a row of
    slab k+1 can become a pivot of slab k (unlike a plain block-Thomas sweep).
    ``factor`` keeps the row permutations and both triangular factors so the
    same factorisation serves any number of right-hand sides (as needed for the
    moments of one expansion point).
    """

    def __init__(self, asm, omega: float):
        self.b, self.nz = asm.b, asm.nz
        self.r, self.c = equilibrate(asm, omega)
        As = (sp.diags(self.r) @ asm.A(omega) @ sp.diags(self.c)).tocsr()
        self._factor(As)

    def _blk(self, As, i, j):
        b = self.b
        if j < 0 or j >= self.nz:
            return np.zeros((b, b), dtype=complex)
        return As[i * b:(i + 1) * b, j * b:(j + 1) * b].toarray().astype(complex)

    def _factor(self, As):
        b, nz = self.b, self.nz
        self.steps = []      # per slab: (perm, L (rows x b), U_kk, U_k,k+1, U_k,k+2)
        # working block row k over block columns k, k+1, k+2
        cur = np.hstack([self._blk(As, 0, 0), self._blk(As, 0, 1), self._blk(As, 0, 2)])
        for k in range(nz):
            if k + 1 < nz:
                nxt = np.hstack([self._blk(As, k + 1, k), self._blk(As, k + 1, k + 1),
                                 self._blk(As, k + 1, k + 2)])
                G = np.vstack([cur, nxt])                       # 2b x 3b
            else:
                G = cur
            P, L, U = la.lu(G[:, :b])                          # G[:, :b] = P L U
            perm = np.argmax(P, axis=0)                        # (P^T G) = G[perm]
            PG = G[perm]
            L11 = L[:b]
            Urest = la.solve_triangular(L11, PG[:b, b:], lower=True, unit_diagonal=True)
            self.steps.append((perm, L, U, Urest))
            if k + 1 < nz:
                L21 = L[b:]
                tail = PG[b:, b:] - L21 @ Urest                 # new block row k+1, cols k+1, k+2
                cur = np.hstack([tail, self._blk(As, k + 1, k + 3)])

    def solve(self, F: np.ndarray) -> np.ndarray:
        b, nz = self.b, self.nz
        F = np.asarray(F, dtype=complex)
        one = F.ndim == 1
        Fs = (self.r[:, None] * (F[:, None] if one else F))
        R = Fs.shape[1]
        y = [Fs[k * b:(k + 1) * b].copy() for k in range(nz)]
        # forward: apply each slab's permutation and unit-lower factor
        for k in range(nz):
            perm, L, U, Urest = self.steps[k]
            if k + 1 < nz:
                rhs = np.vstack([y[k], y[k + 1]])[perm]
                top = la.solve_triangular(L[:b], rhs[:b], lower=True, unit_diagonal=True)
                y[k + 1] = rhs[b:] - L[b:] @ top
                y[k] = top
            else:
                y[k] = la.solve_triangular(L[:b], y[k][perm], lower=True, unit_diagonal=True)
        # backward with U_kk, U_k,k+1, U_k,k+2
        x = [None] * nz
        for k in range(nz - 1, -1, -1):
            perm, L, U, Urest = self.steps[k]
            rhs = y[k].copy()
            if k + 1 < nz:
                rhs -= Urest[:, :b] @ x[k + 1]
            if k + 2 < nz:
                rhs -= Urest[:, b:2 * b] @ x[k + 2]
            x[k] = la.solve_triangular(U, rhs, lower=False)
        X = self.c[:, None] * np.vstack(x)
        return X[:, 0] if one else X


def spl(p: np.ndarray) -> np.ndarray:
    """Sound pressure level re 20 uPa, RMS of a harmonic amplitude |p|."""
    return 20.0 * np.log10(np.abs(p) / (np.sqrt(2.0) * P_REF))


def sweep(asm, freqs_hz, F, rcv_dofs, method: str = "banded"):
    """Full-order sweep: receiver pressures p[f, rcv, col] and their SPL."""
    freqs_hz = np.asarray(freqs_hz, dtype=float)
    out = np.empty((len(freqs_hz), len(rcv_dofs), F.shape[1]), dtype=complex)
    for i, f in enumerate(freqs_hz):
        om = 2.0 * np.pi * f
        if method == "dense":
            x = solve_dense(asm, om, F)
        else:
            x = BlockBandedLU(asm, om).solve(F)
        out[i] = x[rcv_dofs]
    return out, spl(out)


def backward_error(asm, omega: float, x: np.ndarray, f: np.ndarray) -> float:
    """Normwise backward error ||f - A x|| / (||A|| ||x|| + ||f||) of the scaled system."""
    r, c = equilibrate(asm, omega)
    As = sp.diags(r) @ asm.A(omega) @ sp.diags(c)
    y = x / c[:, None] if x.ndim == 2 else x / c
    fs = r[:, None] * f if f.ndim == 2 else r * f
    res = fs - As @ y
    nA = sp.linalg.norm(As, np.inf)
    return float(np.abs(res).max() / (nA * np.abs(y).max() + np.abs(fs).max()))
