"""Pins for the oracle's rational Arnoldi ROM (Sec. 3.3, Eq. 9-11)."""
import numpy as np
import pytest

import workloads as W
from oracle import fem, fom, rom


def _setup(floor):
    w = W.small_model(floor=floor)
    asm = fem.assemble(w.model)
    return w, asm, fem.load_matrix(w.model, w.loads, w.n_rhs), fem.receiver_dofs(w.model, w.receivers)


def _span_gap(A, B):
    """Largest sine of the principal angles between span(A) and span(B)."""
    Qa, _ = np.linalg.qr(A)
    Qb, _ = np.linalg.qr(B)
    return float(np.linalg.norm(Qb - Qa @ (Qa.conj().T @ Qb), 2))


def test_cgs2_orthonormal_and_deflates():
    rng = np.random.default_rng(0)
    X = rng.standard_normal((300, 20)) + 1j * rng.standard_normal((300, 20))
    X[:, 7] = X[:, 2] * (1 + 1j) + 1e-13 * X[:, 3]     # numerically dependent column
    V, acc = rom.cgs2_append(np.zeros((300, 0), complex), X)
    assert V.shape[1] == 19
    assert np.abs(V.conj().T @ V - np.eye(19)).max() < 1e-13
    assert _span_gap(V, np.delete(X, 7, axis=1)) < 1e-10


def test_first_order_basis_spans_explicit_moments():
    """Eq. 10: span{Kt^-1 f, (Kt^-1 M) Kt^-1 f, ...} computed by explicit dense solves."""
    w, asm, F, rc = _setup(floor=False)
    fj = 140.0
    V = rom.build_basis(asm, [fj], 4, F, 100)
    A = asm.A(2 * np.pi * fj).toarray()
    M = asm.M.toarray()
    moments = []
    v = np.linalg.solve(A, F)
    for _ in range(4):
        moments.append(v)
        v = np.linalg.solve(A, M @ v)
    Mm = np.hstack(moments)
    # compare in a column-scaled basis (moment magnitudes grow geometrically)
    Mm = Mm / np.linalg.norm(Mm, axis=0)
    assert V.shape[1] == Mm.shape[1]
    assert _span_gap(V, Mm) < 1e-6


def test_soar_basis_spans_second_order_moments():
    """Eq. 9: r_0 = Kt^-1 f, r_1 = A r_0, r_j = A r_{j-1} + B r_{j-2} with
    A = -Kt^-1 (2 i w_j M + D), B = -Kt^-1 M."""
    w, asm, F, rc = _setup(floor=True)
    assert rom.has_damping_matrix(asm)
    fj = 110.0
    om = 2 * np.pi * fj
    q = 4
    V = rom.build_basis(asm, [fj], q, F[:, :1], 100)
    Kt = asm.A(om).toarray()
    Dt = (2j * om * asm.M + asm.D).toarray()
    M = asm.M.toarray()
    r = [np.linalg.solve(Kt, F[:, 0])]
    r.append(-np.linalg.solve(Kt, Dt @ r[0]))
    for j in range(2, q):
        r.append(-np.linalg.solve(Kt, Dt @ r[j - 1]) - np.linalg.solve(Kt, M @ r[j - 2]))
    R = np.stack([x / np.linalg.norm(x) for x in r], axis=1)
    assert V.shape[1] == q
    assert _span_gap(V, R) < 1e-6


class _Identity:
    """Stands in for the factor of Kt = I (so A = -Dt and B = -M in SOAR)."""

    @staticmethod
    def solve(x):
        return np.array(x, dtype=complex)


class _Pencil:
    def __init__(self, M, D):
        self.M = M
        self.D = D


def _explicit_second_order(Dt, M, u, q):
    """Orthonormal basis of span{r_0..r_{q-1}} (rank-revealing SVD: the sequence is dependent)."""
    r = [u, -Dt @ u]
    for _ in range(2, q):
        r.append(-Dt @ r[-1] - M @ r[-2])
    R = np.stack(r[:q], axis=1)
    U, sv, _ = np.linalg.svd(R, full_matrices=False)
    return U[:, :int((sv > 1e-12 * sv[0]).sum())]


def test_soar_deflation_continues_as_bai_and_su():
    """SOAR's deflation branch (Bai and Su 2005, the reference of Eq. 9): r_1 = A r_0 is parallel
    to r_0, so the step deflates; the recurrence must continue with q = 0 and p = s, because
    r_2 = A r_1 + B r_0 brings in a new direction (B e1 = e2) and r_3 another (A e2 = e3).
    Stopping at the deflation would return span{e1} only.  The explicit sequence fixes the span."""
    n, alpha, gamma = 6, 0.7, 1.9
    D = np.zeros((n, n), complex)
    M = np.zeros((n, n), complex)
    D[0, 0] = -alpha              # A e1 = alpha e1
    M[1, 0] = -1.0                # B e1 = e2
    D[2, 1] = -gamma              # A e2 = gamma e3
    f = np.zeros(n, complex)
    f[0] = -1.0                   # u = -Kt^-1 f = e1
    q = 4
    V = rom._soar(_Pencil(M, D), _Identity(), 0.0, f, q)
    R = _explicit_second_order(D, M, -f, q)
    assert V.shape[1] == 3 == R.shape[1]
    assert np.abs(V.conj().T @ V - np.eye(3)).max() < 1e-14
    assert _span_gap(V, R) < 1e-12


def test_soar_breakdown_when_the_sequence_stays_in_the_span():
    """If after a deflation s also lies in the span of the deflated p vectors, the sequence can
    bring nothing new (here B e1 = 0, so every r_m is a multiple of e1): SOAR stops there."""
    n = 5
    D = np.zeros((n, n), complex)
    M = np.zeros((n, n), complex)
    D[0, 0] = -0.4
    f = np.zeros(n, complex)
    f[0] = 2.0
    V = rom._soar(_Pencil(M, D), _Identity(), 0.0, f, 5)
    R = _explicit_second_order(D, M, -f, 5)
    assert V.shape[1] == 1 == R.shape[1]
    assert _span_gap(V, R) < 1e-12


@pytest.mark.parametrize("floor", [False, True])
def test_rom_interpolates_at_expansion_points(floor):
    """The ROM reproduces the FOM output at every expansion point (moment matching of
    order zero), up to the conditioning of the reduced system."""
    w, asm, F, rc = _setup(floor)
    shifts = [60.0, 150.0, 250.0]
    V = rom.build_basis(asm, shifts, 3, F, 200)
    rm = rom.project(asm, V, F, rc)
    yR = rom.reduced_sweep(rm, shifts)
    y, _ = fom.sweep(asm, shifts, F, rc, method="dense")
    assert rom.relative_error(y, yR).max() < 1e-5
    est = rom.residual_estimate(asm, V, rm, F, shifts)
    assert est.max() < 1e-5


def test_full_basis_reproduces_fom():
    """With V spanning the whole space (k = n) the Galerkin ROM is the FOM."""
    w = W.small_model(nx=3, ny=3, nz=4, Lx=0.3, Ly=0.3, Lz=0.4, floor=True, n_rcv=2)
    asm = fem.assemble(w.model)
    F = fem.load_matrix(w.model, w.loads, w.n_rhs)
    rc = fem.receiver_dofs(w.model, w.receivers)
    rng = np.random.default_rng(3)
    V, _ = rom.cgs2_append(np.zeros((asm.n, 0), complex),
                           rng.standard_normal((asm.n, asm.n)) + 0j)
    assert V.shape[1] == asm.n
    rm = rom.project(asm, V, F, rc)
    yR = rom.reduced_sweep(rm, [80.0, 400.0])
    y, _ = fom.sweep(asm, [80.0, 400.0], F, rc, method="dense")
    # V unitary: A_R = V^H A V keeps the raw (unscaled) conditioning of A, ~1e11 here,
    # so the forward check is loose; the backward error of V x_R (measured in the
    # pressure/displacement-balanced norm of the full system) is the sharper one.
    assert rom.relative_error(y, yR).max() < 1e-4
    for f in (80.0, 400.0):
        om = 2 * np.pi * f
        AR = rm.KR + 1j * om * rm.DR - om ** 2 * rm.MR
        x = V @ np.linalg.solve(AR, rm.fR)
        assert fom.backward_error(asm, om, x, F) < 1e-8


def test_galerkin_orthogonality():
    """V^H (f - A(w) V x_R) = 0 at any frequency."""
    w, asm, F, rc = _setup(floor=True)
    V = rom.build_basis(asm, [70.0, 210.0], 3, F, 100)
    rm = rom.project(asm, V, F, rc)
    om = 2 * np.pi * 133.0
    AR = rm.KR + 1j * om * rm.DR - om ** 2 * rm.MR
    xR = np.linalg.solve(AR, rm.fR)
    r = F - asm.A(om) @ (V @ xR)
    assert np.linalg.norm(V.conj().T @ r) <= 1e-9 * np.linalg.norm(F)


def test_greedy_picks_worst_candidate_and_improves():
    w, asm, F, rc = _setup(floor=False)
    cand = np.arange(40.0, 300.0, 10.0)
    shifts, V, rm, hist = rom.greedy(asm, F, rc, cand, q=3, kmax=200, tol=1e-8, max_shifts=4,
                                     initial_hz=[170.0])
    assert len(shifts) == 4 and len(set(shifts)) == 4
    # every chosen point is interpolated (the estimate collapses there)
    est_at = rom.residual_estimate(asm, V, rm, F, shifts)
    assert est_at.max() < 1e-5
    # the second shift is the argmax of the first estimate away from the first point
    V1 = rom.build_basis(asm, [170.0], 3, F, 200)
    est = rom.residual_estimate(asm, V1, rom.project(asm, V1, F, rc), F, cand)
    allowed = np.abs(cand - 170.0) > 10.0 * 1.0001
    assert shifts[1] == cand[allowed][int(np.argmax(est[allowed]))]


def test_windows_partition_the_band_and_bisect_above_tolerance():
    w, asm, F, rc = _setup(floor=False)
    cand = np.arange(40.0, 300.0, 10.0)
    one = rom.windows(asm, F, rc, cand, q=2, kmax=60, tol=1e3, max_shifts=4, max_windows=8, min_points=3)
    assert len(one) == 1 and one[0]["lo"] == cand[0] and one[0]["hi"] == cand[-1]
    wins = rom.windows(asm, F, rc, cand, q=2, kmax=60, tol=1e-6, max_shifts=4, max_windows=4, min_points=3)
    assert 2 <= len(wins) <= 4
    # ordered, contiguous cover of the candidates, no point in two windows
    covered = [c for win in wins for c in cand if win["lo"] <= c <= win["hi"]]
    assert covered == list(cand)
    # a window above tolerance could not be split further within the budget
    for win in wins:
        npts = sum(1 for c in cand if win["lo"] <= c <= win["hi"])
        assert win["maxest"] <= 1e-6 or npts < 6 or len(wins) == 4


def test_projection_needs_fp64_accuracy():
    """Why the Galerkin projection stays in FP64 (Sec. 3.3, Eq. 11): normwise
    perturbations of K_R, D_R, M_R at the accuracy of a split-precision tensor-core
    product (2^-21, three TF32 products) move the reduced outputs of the config-1 model
    by far more than 0.1 dB, while FP64-level perturbations do not."""
    import copy
    w = W.config1()
    asm = fem.assemble(w.model)
    F = fem.load_matrix(w.model, w.loads, w.n_rhs)
    rc = fem.receiver_dofs(w.model, w.receivers)
    V = rom.build_basis(asm, [40.0, 90.0, 140.0, 185.0], 8, F, 200)
    rm = rom.project(asm, V, F, rc)
    freqs = np.arange(20.0, 200.5, 1.0)
    y0 = rom.reduced_sweep(rm, freqs)
    rng = np.random.default_rng(0)

    def worst_db(eps):
        r2 = copy.copy(rm)
        for attr in ("KR", "DR", "MR"):
            A = getattr(rm, attr)
            if np.abs(A).max() == 0:
                continue
            E = rng.standard_normal(A.shape) + 1j * rng.standard_normal(A.shape)
            setattr(r2, attr, A + E * (eps * np.linalg.norm(A, 2) / np.linalg.norm(E, 2)))
        y = rom.reduced_sweep(r2, freqs)
        return float(np.abs(20.0 * np.log10(np.abs(y) / np.abs(y0))).max())

    assert worst_db(2.0 ** -53) < 1e-6
    assert worst_db(2.0 ** -21) > 0.1


def test_full_residual_vanishes_at_expansion_points_and_with_a_complete_basis():
    """The lifted reduced solution solves the full system at an expansion point (the moment
    block contains A(w_j)^-1 f) and at every frequency when V spans C^n, up to the rounding
    of the ill-conditioned reduced solve (unscaled residual ~1e-8 here, against ~1e-12 for
    a direct FP64 solve of the full system); between the points it does not."""
    w, asm, F, rc = _setup(floor=True)
    shifts = [70.0, 210.0]
    V = rom.build_basis(asm, shifts, 3, F, 200)
    rm = rom.project(asm, V, F, rc)
    r = rom.full_residual(asm, V, rm, F, [70.0, 140.0, 210.0])
    assert r.shape == (3, F.shape[1])
    assert r[0].max() < 1e-6 and r[2].max() < 1e-6
    assert r[1].max() > 1e3 * max(r[0].max(), r[2].max())
    Q, _ = np.linalg.qr(np.random.default_rng(2).standard_normal((asm.n, asm.n)) + 0j)
    full = rom.project(asm, Q, F, rc)
    assert rom.full_residual(asm, Q, full, F, [140.0]).max() < 1e-6


def test_windows_reuse_the_enclosing_windows_points():
    """With reuse, the two halves of a bisected window start from the whole window's
    expansion points in their bands, in the order they were chosen; without reuse they
    start from their own quarter midpoints.  Both partitions cover the band."""
    w, asm, F, rc = _setup(floor=False)
    cand = np.arange(40.0, 300.0, 10.0)
    kw = dict(q=2, kmax=60, tol=1e-6, max_shifts=4, max_windows=2, min_points=3)
    quarter = [float(cand[int(np.argmin(np.abs(cand - (cand[0] + (cand[-1] - cand[0]) * (qq + 0.5) / 4.0))))])
               for qq in range(4)]
    root, _, _, hist = rom.greedy(asm, F, rc, cand, 2, 60, 1e-6, 4, initial_hz=quarter)
    assert hist[-1] > 1e-6   # the whole band is bisected
    for reuse in (False, True):
        wins = rom.windows(asm, F, rc, cand, reuse=reuse, **kw)
        assert len(wins) == 2
        covered = [x for win in wins for x in cand if win["lo"] <= x <= win["hi"]]
        assert covered == list(cand)
        for win in wins:
            inband = [sh for sh in root if win["lo"] <= sh <= win["hi"]]
            if reuse:
                assert inband and win["reused"] == len(inband)
                assert win["shifts"][:len(inband)] == inband
            else:
                assert win["reused"] == 0
