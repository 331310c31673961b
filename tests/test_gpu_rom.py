"""Rational Arnoldi ROM on the GPU against the oracle's ROM with the same
expansion points and moment counts (Sec. 3.3, Eq. 9-11): reduced outputs agree to
1e-6 (the Galerkin output does not depend on which basis of the Krylov space is
used), the basis is orthonormal, and the ROM interpolates the full-order model at
the expansion points."""
import numpy as np
import pytest

import workloads as W
from gpu_util import need_cuda, rel
from oracle import fem, fom, rom

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("floor", [False, True])
def test_rom_matches_oracle_rom(floor):
    torch = need_cuda()
    from paper_2310_04734_gb300 import api
    w = W.small_model(floor=floor)
    spec = w.model
    shifts = [60.0, 150.0, 250.0]
    q = 3
    model = api.fsi_assemble(spec)
    F = api.dense_loads(spec, w.loads, w.n_rhs)
    rcv = torch.tensor(api.receiver_dofs(spec, w.receivers), device="cuda")
    V = api.rom_build(model, shifts, q, F, kmax=200, precision="fp32_ir", tol=1e-12, max_refine=30)
    Vh = V.cpu().numpy()
    assert np.abs(Vh.conj().T @ Vh - np.eye(Vh.shape[1])).max() < 1e-12
    rm = api.rom_project(model, V, F, rcv)
    freqs = np.array([45.0, 60.0, 100.0, 150.0, 200.0, 250.0, 280.0])
    p, spl = api.rom_sweep(rm, freqs, batch=4)
    asm = fem.assemble(spec)
    Fo = fem.load_matrix(spec, w.loads, w.n_rhs)
    rco = fem.receiver_dofs(spec, w.receivers)
    Vo = rom.build_basis(asm, shifts, q, Fo, 200)
    assert Vo.shape[1] == Vh.shape[1]
    yR = rom.reduced_sweep(rom.project(asm, Vo, Fo, rco), freqs)
    pg = p.cpu().numpy()
    assert rel(pg, yR) <= 1e-6
    # interpolation at the expansion points (vs the full-order oracle)
    y, _ = fom.sweep(asm, shifts, Fo, rco, method="dense")
    idx = [list(freqs).index(s) for s in shifts]
    assert rom.relative_error(y, pg[idx]).max() < 1e-5


@pytest.mark.parametrize("floor", [False, True])
def test_rom_residual_check_matches_oracle(floor):
    """FP64 full-order residual of the lifted reduced solutions (CSR residual kernel)
    against the oracle's explicit residual with its own basis of the same Krylov space;
    batch 3 over 7 frequencies leaves a ragged last batch."""
    torch = need_cuda()
    from paper_2310_04734_gb300 import api
    w = W.small_model(floor=floor)
    spec = w.model
    shifts = [60.0, 150.0, 250.0]
    q = 3
    model = api.fsi_assemble(spec)
    F = api.dense_loads(spec, w.loads, w.n_rhs)
    rcv = torch.tensor(api.receiver_dofs(spec, w.receivers), device="cuda")
    V = api.rom_build(model, shifts, q, F, kmax=200, precision="fp32_ir", tol=1e-12, max_refine=30)
    rm = api.rom_project(model, V, F, rcv)
    freqs = np.array([45.0, 60.0, 100.0, 150.0, 200.0, 250.0, 280.0])
    got = api.rom_residual_check(model, V, rm, F, freqs, batch=3)
    asm = fem.assemble(spec)
    Fo = fem.load_matrix(spec, w.loads, w.n_rhs)
    Vo = rom.build_basis(asm, shifts, q, Fo, 200)
    ref = rom.full_residual(asm, Vo, rom.project(asm, Vo, Fo, fem.receiver_dofs(spec, w.receivers)), Fo, freqs)
    assert got.shape == ref.shape
    # residuals span many decades; at the expansion points both sit at the reduced solve's rounding
    assert np.all(np.abs(got - ref) <= 1e-3 * ref + 1e-6), (got, ref)
    idx = [list(freqs).index(s) for s in shifts]
    assert got[idx].max() < 1e-5


def test_projection_matches_oracle_matrices():
    torch = need_cuda()
    from paper_2310_04734_gb300 import api
    w = W.small_model(floor=True)
    spec = w.model
    model = api.fsi_assemble(spec)
    asm = fem.assemble(spec)
    rng = np.random.default_rng(4)
    Vn, _ = np.linalg.qr(rng.standard_normal((asm.n, 37)) + 1j * rng.standard_normal((asm.n, 37)))
    F = api.dense_loads(spec, w.loads, w.n_rhs)
    rcv = torch.tensor(api.receiver_dofs(spec, w.receivers), device="cuda")
    rm = api.rom_project(model, torch.tensor(Vn, device="cuda"), F, rcv)
    ref = rom.project(asm, Vn, fem.load_matrix(spec, w.loads, w.n_rhs), fem.receiver_dofs(spec, w.receivers))
    for got, exp in ((rm.KR, ref.KR), (rm.DR, ref.DR), (rm.MR, ref.MR), (rm.fR, ref.fR), (rm.CR, ref.CR)):
        g = got.cpu().numpy()
        assert np.abs(g - exp).max() <= 1e-12 * max(np.abs(exp).max(), 1e-300)


@pytest.mark.parametrize("floor", [False, True])
def test_greedy_matches_oracle_greedy(floor):
    """Greedy expansion points on the GPU (Gram-block residual estimate) against the
    oracle's greedy (explicit FP64 residuals): same points, same largest estimate per
    round, same estimates on the candidate grid, same reduced outputs."""
    torch = need_cuda()
    from paper_2310_04734_gb300 import api
    w = W.small_model(floor=floor)
    spec = w.model
    model = api.fsi_assemble(spec)
    F = api.dense_loads(spec, w.loads, w.n_rhs)
    rcv = torch.tensor(api.receiver_dofs(spec, w.receivers), device="cuda")
    cand = np.arange(40.0, 300.0, 10.0)
    # FP64 moments: this small ROM is far from converged (estimates ~1), so its outputs
    # amplify basis rounding; the FP32-factor path is checked in the tests above
    g = api.rom_greedy(model, F, rcv, cand, q=3, kmax=200, max_shifts=4, tol=1e-8, init_hz=[170.0],
                       precision="fp64", max_refine=5, refine_tol=1e-13)
    asm = fem.assemble(spec)
    Fo = fem.load_matrix(spec, w.loads, w.n_rhs)
    rco = fem.receiver_dofs(spec, w.receivers)
    shifts, Vo, rm, hist = rom.greedy(asm, Fo, rco, cand, q=3, kmax=200, tol=1e-8, max_shifts=4,
                                      initial_hz=[170.0])
    print("greedy shifts gpu", g.shifts_hz.tolist(), "oracle", shifts, "hist", g.history.tolist(), hist)
    assert g.shifts_hz.tolist() == shifts
    assert np.allclose(g.history, hist, rtol=1e-4, atol=0)
    est_o = rom.residual_estimate(asm, Vo, rm, Fo, cand)
    big = est_o > 1e-6
    assert np.abs(g.est[big] / est_o[big] - 1).max() < 1e-3
    assert np.all(g.est[~big] < 1e-5)
    # the Gram-block projection equals the oracle's projection of the same basis
    Vg = g.V.cpu().numpy()
    ref = rom.project(asm, Vg, Fo, rco)
    for got, exp in ((g.rom.KR, ref.KR), (g.rom.DR, ref.DR), (g.rom.MR, ref.MR), (g.rom.fR, ref.fR),
                     (g.rom.CR, ref.CR)):
        assert np.abs(got.cpu().numpy() - exp).max() <= 1e-12 * max(np.abs(exp).max(), 1e-300)
    # this 24-column ROM is poor away from its points (estimates ~1), so its outputs are
    # compared through the same basis, and against the full-order model at the points
    freqs = np.array([45.0, 101.0, 222.0, 290.0])
    p, _ = api.rom_sweep(g.rom, freqs, batch=4)
    assert rel(p.cpu().numpy(), rom.reduced_sweep(ref, freqs)) <= 1e-8
    ps, _ = api.rom_sweep(g.rom, shifts, batch=4)
    y, _ = fom.sweep(asm, shifts, Fo, rco, method="dense")
    assert rom.relative_error(y, ps.cpu().numpy()).max() < 1e-5


@pytest.mark.parametrize("reuse", [False, True])
def test_windows_match_oracle_windows(reuse):
    """Local ROM windows on the GPU against the oracle's windows: same partition, same
    points per window (and as many reused from enclosing windows), same final estimates,
    same reduced outputs per window."""
    torch = need_cuda()
    from paper_2310_04734_gb300 import api
    w = W.small_model(floor=False)
    spec = w.model
    model = api.fsi_assemble(spec)
    F = api.dense_loads(spec, w.loads, w.n_rhs)
    rcv = torch.tensor(api.receiver_dofs(spec, w.receivers), device="cuda")
    cand = np.arange(40.0, 300.0, 10.0)
    g = api.rom_windows(model, F, rcv, cand, q=2, kmax=60, max_shifts=4, tol=1e-6, max_windows=4, min_points=3,
                        precision="fp64", max_refine=5, refine_tol=1e-13, reuse=reuse)
    asm = fem.assemble(spec)
    Fo = fem.load_matrix(spec, w.loads, w.n_rhs)
    rco = fem.receiver_dofs(spec, w.receivers)
    wins = rom.windows(asm, Fo, rco, cand, q=2, kmax=60, tol=1e-6, max_shifts=4, max_windows=4, min_points=3,
                       reuse=reuse)
    print("windows gpu", g.lo.tolist(), g.hi.tolist(), g.maxest.tolist(), "oracle",
          [(x["lo"], x["hi"], x["maxest"]) for x in wins])
    assert g.lo.tolist() == [x["lo"] for x in wins] and g.hi.tolist() == [x["hi"] for x in wins]
    assert g.nshift.tolist() == [len(x["shifts"]) for x in wins]
    assert g.nreused.tolist() == [x["reused"] for x in wins]
    assert (g.nreused.sum() > 0) == reuse
    # estimates near the rounding level of a solve (windows whose every candidate is an
    # expansion point) carry no digits; compare the others
    mo = np.array([x["maxest"] for x in wins])
    big = mo > 1e-5
    assert np.allclose(g.maxest[big], mo[big], rtol=1e-2, atol=0) and np.all(g.maxest[~big] < 1e-5)
    freqs = np.array([42.0, 95.0, 151.0, 208.0, 263.0, 297.0])
    p, _ = api.rom_windows_sweep(g, freqs, batch=4)
    ref = []
    for f in freqs:
        x = next((x for x in wins if x["lo"] <= f <= x["hi"]), None)
        if x is None:   # between windows: the nearer one
            x = min(wins, key=lambda x: min(abs(f - x["lo"]), abs(f - x["hi"])))
        ref.append(rom.reduced_sweep(x["rm"], [f])[0])
    # poorly converged windows amplify basis rounding in their outputs (as in the greedy test)
    assert rel(p.cpu().numpy(), np.array(ref)) <= 1e-4


def _small_rom(floor=True):
    torch = need_cuda()
    from paper_2310_04734_gb300 import api
    w = W.small_model(floor=floor)
    spec = w.model
    model = api.fsi_assemble(spec)
    F = api.dense_loads(spec, w.loads, w.n_rhs)
    rcv = torch.tensor(api.receiver_dofs(spec, w.receivers), device="cuda")
    shifts = [60.0, 150.0, 250.0]
    V = api.rom_build(model, shifts, 3, F, kmax=200, precision="fp32_ir", tol=1e-12, max_refine=30)
    return api, w, model, F, rcv, shifts, V, api.rom_project(model, V, F, rcv)


def test_rom_save_load_round_trip_on_the_device(tmp_path):
    """A reduced model (matrices, expansion points, basis) written from device buffers and read
    back gives bit-identical buffers and the same reduced sweep."""
    torch = need_cuda()
    api, w, model, F, rcv, shifts, V, rm = _small_rom()
    path = str(tmp_path / "small.fsirom")
    api.rom_save(path, rm, shifts, V=V, band=(20.0, 300.0))
    r2, sh2, V2, band = api.rom_load(path)
    for a, b in ((rm.KR, r2.KR), (rm.DR, r2.DR), (rm.MR, r2.MR), (rm.fR, r2.fR), (rm.CR, r2.CR), (V, V2)):
        assert torch.equal(a.contiguous(), b.contiguous())
    assert list(sh2) == shifts and band == (20.0, 300.0)
    freqs = np.array([45.0, 133.0, 280.0])
    p1, _ = api.rom_sweep(rm, freqs, batch=3)
    p2, _ = api.rom_sweep(r2, freqs, batch=3)
    assert torch.equal(p1, p2)


def test_rom_sweep_fp32_refined_matches_fp64():
    """rom_sweep with precision FSI_FP32_IR (FP32 LU refined against the FP64 residual, FP64
    re-solve where the refinement stalls) against the FP64 reduced LU and the oracle's ROM."""
    torch = need_cuda()
    api, w, model, F, rcv, shifts, V, rm = _small_rom()
    freqs = np.linspace(30.0, 290.0, 27)
    p64, spl64 = api.rom_sweep(rm, freqs, batch=8)
    p32, spl32, fb = api.rom_sweep(rm, freqs, batch=8, precision="fp32_ir", return_fp64=True)
    a, b = p32.cpu().numpy(), p64.cpu().numpy()
    errs = np.array([rel(a[i], b[i]) for i in range(len(freqs))])
    print("fp32_ir vs fp64 reduced sweep: max %.2e, FP64 re-solves %d" % (errs.max(), int(fb.sum())))
    assert errs.max() <= 1e-6
    assert np.abs(spl32.cpu().numpy() - spl64.cpu().numpy()).max() <= 1e-5


def test_check_and_resolve_replaces_failing_frequencies_by_full_order():
    """rom_check_resolve judges every frequency by the full-order FP64 residual of the lifted
    reduced solution.  With res_tol = 0 every frequency fails the check (a planted failure) and
    its outputs must become the full-order ones; with a loose tolerance nothing changes."""
    torch = need_cuda()
    api, w, model, F, rcv, shifts, V, rm = _small_rom()
    freqs = np.array([45.0, 97.0, 150.0, 212.0, 280.0])
    p, spl = api.rom_sweep(rm, freqs, batch=5)
    keep_p, keep_spl = p.clone(), spl.clone()
    ref = api.rom_residual_check(model, V, rm, F, freqs)
    loose = 2.0 * ref.max()                   # above every residual: nothing fails the check
    rel_l, res_l, n_l = api.rom_check_resolve(model, V, rm, F, rcv, freqs, p, spl, res_tol=loose)
    assert n_l == 0 and not res_l.any() and torch.equal(p, keep_p) and torch.equal(spl, keep_spl)
    assert np.allclose(rel_l, ref, rtol=1e-12, atol=0)
    # a tolerance between the residuals re-solves exactly the frequencies above it: placed in the
    # widest relative gap between two of them, since the call recomputes the residuals and norms
    # reduced with atomics may differ in the last bits from those of rom_residual_check
    r = np.sort(ref.max(axis=1))
    g = int(np.argmax(r[1:] / r[:-1]))
    mid = float(np.sqrt(r[g] * r[g + 1]))
    _, res_m, n_m = api.rom_check_resolve(model, V, rm, F, rcv, freqs, p.clone(), spl.clone(), res_tol=mid)
    assert n_m == int((ref.max(axis=1) > mid).sum()) and (res_m == (ref.max(axis=1) > mid)).all()
    rel_0, res_0, n_0 = api.rom_check_resolve(model, V, rm, F, rcv, freqs, p, spl, res_tol=0.0)
    assert n_0 == len(freqs) and res_0.all()
    full = api.frf_sweep_full(model, freqs, F, rcv, precision="fp32_ir", batch=5, max_refine=60, tol=1e-10)
    # the same kernels and batch as the call's re-solve (sums of atomically reduced norms may
    # round differently from run to run)
    assert rel(p.cpu().numpy(), full.p.cpu().numpy()) <= 1e-11
    assert np.abs(spl.cpu().numpy() - full.spl.cpu().numpy()).max() <= 1e-9
    asm = fem.assemble(w.model)
    y, _ = fom.sweep(asm, freqs, fem.load_matrix(w.model, w.loads, w.n_rhs), fem.receiver_dofs(w.model, w.receivers),
                     method="dense")
    assert rel(p.cpu().numpy(), y) <= 1e-8


@pytest.mark.parametrize("precision", ["fp32_ir", "bf16x6_ir"])
def test_batched_expansion_points_match_one_at_a_time(precision):
    """Eq. 10 moments of several expansion points factored and solved together (batch_shifts)
    give the same basis span, hence the same reduced outputs, as one point at a time, and
    both match the oracle's ROM; the tensor-core factor (BF16x6) serves the moments too."""
    torch = need_cuda()
    from paper_2310_04734_gb300 import api
    w = W.small_model(floor=False)
    spec = w.model
    model = api.fsi_assemble(spec)
    F = api.dense_loads(spec, w.loads, w.n_rhs)
    rcv = torch.tensor(api.receiver_dofs(spec, w.receivers), device="cuda")
    shifts, q = [60.0, 150.0, 250.0, 110.0], 3
    freqs = np.array([45.0, 97.0, 133.0, 210.0, 280.0])
    outs = []
    for bs in (1, 3, 4):
        V = api.rom_build(model, shifts, q, F, kmax=200, precision=precision, tol=1e-12, max_refine=30,
                          batch_shifts=bs)
        p, _ = api.rom_sweep(api.rom_project(model, V, F, rcv), freqs, batch=5)
        outs.append((V.shape[1], p.cpu().numpy()))
    assert outs[0][0] == outs[1][0] == outs[2][0]
    assert rel(outs[1][1], outs[0][1]) <= 1e-8 and rel(outs[2][1], outs[0][1]) <= 1e-8
    asm = fem.assemble(spec)
    Fo = fem.load_matrix(spec, w.loads, w.n_rhs)
    yR = rom.reduced_sweep(rom.project(asm, rom.build_basis(asm, shifts, q, Fo, 200), Fo,
                                       fem.receiver_dofs(spec, w.receivers)), freqs)
    assert rel(outs[1][1], yR) <= 1e-6
