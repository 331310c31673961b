"""Pins for the oracle's full-order solution x(w) = A(w)^-1 f (Sec. 2, Eq. 1; Eq. 8).

Independent checks: two different direct solvers agree; both are backward
stable; transfer functions obey acoustic-structural reciprocity (a property of
the coupled operator that a sign or transpose slip in a coupling block breaks);
the SPL convention.
"""
import dataclasses

import numpy as np
import pytest
import scipy.sparse as sp

import workloads as W
from oracle import fem, fom


@pytest.fixture(scope="module")
def small():
    w = W.small_model()
    asm = fem.assemble(w.model)
    return w, asm, fem.load_matrix(w.model, w.loads, w.n_rhs), fem.receiver_dofs(w.model, w.receivers)


@pytest.fixture(scope="module")
def cfg1():
    w = W.config1()
    asm = fem.assemble(w.model)
    return w, asm, fem.load_matrix(w.model, w.loads, w.n_rhs), fem.receiver_dofs(w.model, w.receivers)


@pytest.mark.parametrize("f_hz", [31.0, 97.5, 233.0])
def test_dense_equals_block_banded_small(small, f_hz):
    w, asm, F, rc = small
    om = 2 * np.pi * f_hz
    xd = fom.solve_dense(asm, om, F)
    xb = fom.BlockBandedLU(asm, om).solve(F)
    assert np.linalg.norm(xd - xb) <= 1e-10 * np.linalg.norm(xd)
    assert fom.backward_error(asm, om, xd, F) < 1e-14
    assert fom.backward_error(asm, om, xb, F) < 1e-14


@pytest.mark.parametrize("f_hz", [20.0, 88.0, 171.0, 200.0])
def test_dense_equals_block_banded_config1(cfg1, f_hz):
    w, asm, F, rc = cfg1
    om = 2 * np.pi * f_hz
    xd = fom.solve_dense(asm, om, F)
    xb = fom.BlockBandedLU(asm, om).solve(F)
    assert np.linalg.norm(xd[rc] - xb[rc]) <= 1e-10 * np.linalg.norm(xd[rc])
    assert fom.backward_error(asm, om, xb, F) < 1e-14


def test_unscaled_dense_solve_is_the_same_definition(small):
    """The scaling is exact algebra: LAPACK on the raw matrix gives the same x (to its own,
    worse, conditioning)."""
    w, asm, F, rc = small
    om = 2 * np.pi * 77.0
    x_raw = np.linalg.solve(asm.A(om).toarray(), F)
    x = fom.solve_dense(asm, om, F)
    assert np.linalg.norm(x_raw[rc] - x[rc]) <= 1e-7 * np.linalg.norm(x[rc])


def _reciprocity_gap(asm, spec, f_hz):
    num = fem.Numbering(spec)
    om = 2 * np.pi * f_hz
    a = num.s(3, 2, 0)          # shell w-DoF (not on the supported ends)
    b = num.p(2, 1, 3)          # interior pressure DoF
    ea = np.zeros((asm.n, 1), complex); ea[a] = 1.0
    eb = np.zeros((asm.n, 1), complex); eb[b] = 1.0
    H_pF = fom.solve_dense(asm, om, ea)[b, 0]      # pressure at b per unit force at a
    H_wQ = fom.solve_dense(asm, om, eb)[a, 0]      # displacement at a per unit fluid source at b
    return abs(H_pF - spec.rho * om ** 2 * H_wQ) / abs(H_pF)


@pytest.mark.parametrize("f_hz", [45.0, 160.0])
def test_reciprocity(small, f_hz):
    """S A T is complex symmetric (S = diag(I, -1/(rho w^2)), T = diag(I, -I)), hence
    H_{p_b <- F_a} = rho w^2 H_{w_a <- Q_b} exactly."""
    w, asm, F, rc = small
    assert _reciprocity_gap(asm, w.model, f_hz) < 1e-9


def test_reciprocity_catches_a_planted_coupling_sign_error(small):
    """Planting a sign error in the fluid-structure mass block (rho C^T -> -rho C^T)
    must break the reciprocity pin, so the pin does test the coupling."""
    w, asm, F, rc = small
    fl = asm.is_fluid
    M = asm.M.tolil()
    rows, cols = np.where(np.outer(fl, ~fl) & (asm.M.toarray() != 0))
    for r, c in zip(rows, cols):
        M[r, c] = -M[r, c]
    bad = dataclasses.replace(asm, M=M.tocsr())
    assert _reciprocity_gap(bad, w.model, 45.0) > 1e-3


def test_uncoupled_limit(small):
    """With the coupling removed, a shell load produces no pressure, and the shell
    response equals the shell-only solve."""
    w, asm, F, rc = small
    fl = asm.is_fluid
    keep = sp.diags(1.0 * fl) @ asm.K @ sp.diags(1.0 * fl) + sp.diags(1.0 * ~fl) @ asm.K @ sp.diags(1.0 * ~fl)
    keepM = sp.diags(1.0 * fl) @ asm.M @ sp.diags(1.0 * fl) + sp.diags(1.0 * ~fl) @ asm.M @ sp.diags(1.0 * ~fl)
    dec = dataclasses.replace(asm, K=keep.tocsr(), M=keepM.tocsr())
    om = 2 * np.pi * 120.0
    x = fom.solve_dense(dec, om, F)
    assert np.abs(x[fl]).max() == 0.0
    sh = ~fl
    As = dec.A(om)[sh][:, sh].toarray()
    xs = np.linalg.solve(As, F[sh])
    assert np.linalg.norm(x[sh] - xs) <= 1e-9 * np.linalg.norm(xs)


def test_spl_convention():
    pref = np.sqrt(2.0) * 2e-5
    assert np.allclose(fom.spl(np.array([pref, 10 * pref, 1j * pref])), [0.0, 20.0, 0.0])


def test_sweep_shapes(small):
    w, asm, F, rc = small
    p, L = fom.sweep(asm, [50.0, 60.0], F, rc, method="dense")
    assert p.shape == (2, len(rc), w.n_rhs) and L.shape == p.shape


def test_golden_fixture_reproduces_from_the_oracle():
    """tests/golden/cfg1_fom.json (written by tests/golden/make_golden.py from the oracle
    only) matches a fresh oracle solve at sampled frequencies, for the same workload,
    receivers and frequency grid."""
    import json
    import os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "cfg1_fom.json")))
    w = W.config1()
    assert g["workload"] == w.name and g["freqs_hz"] == w.freqs_hz.tolist()
    assert [tuple(r) for r in g["receivers"]] == [tuple(r) for r in w.receivers]
    asm = fem.assemble(w.model)
    F = fem.load_matrix(w.model, w.loads, w.n_rhs)
    rc = fem.receiver_dofs(w.model, w.receivers)
    idx = [0, 57, 180]
    p, _ = fom.sweep(asm, w.freqs_hz[idx], F, rc, method="dense")
    stored = np.array(g["p_re"])[idx] + 1j * np.array(g["p_im"])[idx]
    assert np.abs(p - stored).max() <= 1e-12 * np.abs(stored).max()
    assert all(k >= 1.0 for k in g["kappa1_scaled"])
