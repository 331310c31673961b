"""Full-order sweep on the GPU against the oracle (paper Sec. 2, Eq. 1; Eq. 8).

FP64 path: relative 2-norm error on the receivers <= max(1e-10, 10 kappa u)
per frequency, kappa the oracle's 1-norm condition estimate of the scaled
system.  The GPU's C++ assembly and the oracle's quadrature differ by a few
ulps per entry, which alone moves the solution by ~kappa u (up to 3e-10 at
27-38 Hz on config 1, kappa ~ 1e6); at most frequencies the agreement is
~1e-11.  Mixed path (FP32 factor + FP64 GMRES refinement): <= 1e-6 relative
and <= 0.1 dB at a 1e-8 residual target, and the FP64 bound at a tight one.
"""
import json
import os

import numpy as np
import pytest

import workloads as W
from gpu_util import db_err, need_cuda, rel
from oracle import fem, fom

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


U64 = np.finfo(np.float64).eps / 2


def _golden_cfg1():
    g = json.load(open(os.path.join(HERE, "golden", "cfg1_fom.json")))
    return (np.array(g["freqs_hz"]), np.array(g["p_re"]) + 1j * np.array(g["p_im"]),
            np.array(g["kappa1_scaled"]))


def _fp64_bound(kappa):
    return np.maximum(1e-10, 10.0 * np.asarray(kappa) * U64)


def _dense_kappa(asm, freqs):
    import scipy.sparse as sp
    out = []
    for f in freqs:
        om = 2 * np.pi * f
        r, c = fom.equilibrate(asm, om)
        As = (sp.diags(r) @ asm.A(om) @ sp.diags(c)).toarray()
        out.append(np.linalg.cond(As, 1))
    return np.array(out)


def _setup(w):
    torch = need_cuda()
    from paper_2310_04734_gb300 import api
    model = api.fsi_assemble(w.model)
    F = api.dense_loads(w.model, w.loads, w.n_rhs)
    rcv = torch.tensor(api.receiver_dofs(w.model, w.receivers), device="cuda")
    return api, model, F, rcv


def _per_freq_rel(p, y):
    return np.array([rel(p[i], y[i]) for i in range(len(y))])


def test_cfg1_fp64_all_181_frequencies_vs_golden():
    w = W.config1()
    api, model, F, rcv = _setup(w)
    freqs, y, kappa = _golden_cfg1()
    res = api.frf_sweep_full(model, freqs, F, rcv, precision="fp64", batch=64, max_refine=2, tol=1e-15,
                             allow_noconv=True)
    p = res.p.cpu().numpy()
    e = _per_freq_rel(p, y)
    print("fp64 vs oracle: max %.3e median %.3e at %.1f Hz" % (e.max(), np.median(e), freqs[np.argmax(e)]))
    assert (e <= _fp64_bound(kappa)).all(), (e.max(), freqs[np.argmax(e / _fp64_bound(kappa))])
    assert np.median(e) <= 1e-10
    assert res.relres.max() < 1e-9        # FP64 rounding floor of the scaled residual near resonances


@pytest.mark.parametrize("precision", ["fp32_ir", "bf16x6_ir"])
def test_cfg1_mixed_all_181_frequencies_vs_golden(precision):
    """Config 3: the config-1 model factored in FP32 (SIMT) or with the long trailing updates
    on the tensor cores (BF16x6: three-plane BF16 splits, FP32-level), refined by FP64 GMRES
    to 1e-8."""
    w = W.config3()
    api, model, F, rcv = _setup(w)
    freqs, y, kappa = _golden_cfg1()
    res = api.frf_sweep_full(model, freqs, F, rcv, precision=precision, batch=64, max_refine=40, tol=1e-8)
    p = res.p.cpu().numpy()
    assert _per_freq_rel(p, y).max() <= 1e-6
    assert db_err(p, y) <= 0.1
    assert res.relres.max() <= 1e-8 and res.stats.n_unconverged == 0
    print("mixed iterations: max %d mean %.2f" % (res.iters.max(), res.iters.mean()))
    assert res.iters.max() <= 12
    tight = api.frf_sweep_full(model, freqs, F, rcv, precision=precision, batch=64, max_refine=40, tol=1e-11,
                               allow_noconv=True)
    assert (_per_freq_rel(tight.p.cpu().numpy(), y) <= _fp64_bound(kappa)).all()


def test_cfg3_plain_bf16_factor_is_a_weak_preconditioner():
    """Config 3's BF16 variant: the config-1 model factored with plain BF16 products (one plane,
    FP32 accumulation) and refined by FP64 GMRES.  At 8 unit roundoff bits the factor's error,
    times the condition numbers of these systems, is far above one, so the refinement either
    fails within 60 steps or needs several times the steps of the three-plane factor; the
    frequencies it does converge at must still agree with the oracle."""
    w = W.config3()
    api, model, F, rcv = _setup(w)
    freqs, y, kappa = _golden_cfg1()
    sel = np.arange(0, len(freqs), 12)            # 16 frequencies across the band
    f, y = freqs[sel], y[sel]
    kw = dict(batch=16, max_refine=60, tol=1e-8, allow_noconv=True)
    six = api.frf_sweep_full(model, f, F, rcv, precision="bf16x6_ir", **kw)
    one = api.frf_sweep_full(model, f, F, rcv, precision="bf16_ir", **kw)
    it6, it1 = six.iters, one.iters
    conv = one.relres <= 1e-8
    print("plain BF16: %d of %d converged, GMRES steps mean %.1f (BF16x6 %.1f)"
          % (conv.sum(), len(f), np.mean(it1), np.mean(it6)))
    assert six.stats.n_unconverged == 0
    assert one.stats.n_unconverged > 0 or np.mean(it1) >= 3.0 * np.mean(it6)
    p1 = one.p.cpu().numpy()
    assert all(rel(p1[i], y[i]) <= 1e-6 for i in np.flatnonzero(conv))


@pytest.mark.parametrize("precision,refine", [("fp64", "ir"), ("fp32_ir", "gmres"), ("fp32_ir", "ir")])
def test_small_model_with_floor_impedance_ragged_batches(precision, refine):
    """D != 0 (floor impedance); nf = 7 with batch 3 leaves a ragged last batch."""
    w = W.small_model(floor=True, n_loads=2, n_rcv=4)
    api, model, F, rcv = _setup(w)
    freqs = np.array([33.0, 71.5, 110.0, 190.0, 251.0, 333.0, 410.0])
    res = api.frf_sweep_full(model, freqs, F, rcv, precision=precision, batch=3, max_refine=40, tol=1e-11,
                             allow_noconv=True, refine=refine)
    asm = fem.assemble(w.model)
    y, L = fom.sweep(asm, freqs, fem.load_matrix(w.model, w.loads, w.n_rhs),
                     fem.receiver_dofs(w.model, w.receivers), method="dense")
    p = res.p.cpu().numpy()
    assert (_per_freq_rel(p, y) <= _fp64_bound(_dense_kappa(asm, freqs))).all()
    assert np.abs(res.spl.cpu().numpy() - L).max() <= 1e-6


def test_many_load_columns_and_host_io():
    """nrhs = 6 (> one 4-column solve group) through the host-buffer entry path."""
    w = W.small_model(nx=4, ny=5, nz=7, floor=True, n_loads=6, n_rcv=3, cfg_id=77)
    api, model, F, rcv = _setup(w)
    freqs = np.array([55.0, 140.0, 260.0])
    res = api.frf_sweep_full(model, freqs, F.cpu().numpy(), rcv.cpu().numpy(), precision="fp32_ir",
                             batch=2, max_refine=40, tol=1e-11, host_io=True, allow_noconv=True)
    asm = fem.assemble(w.model)
    y, _ = fom.sweep(asm, freqs, fem.load_matrix(w.model, w.loads, w.n_rhs),
                     fem.receiver_dofs(w.model, w.receivers), method="dense")
    assert (_per_freq_rel(res.p, y) <= _fp64_bound(_dense_kappa(asm, freqs))).all()


def test_minimal_slab_count():
    """nz = 3: the first, a middle and the last slab step only."""
    w = W.small_model(nx=3, ny=4, nz=3, Lx=0.3, Ly=0.4, Lz=0.3, floor=True, n_loads=1, n_rcv=1, cfg_id=5)
    api, model, F, rcv = _setup(w)
    freqs = np.array([100.0, 700.0])
    res = api.frf_sweep_full(model, freqs, F, rcv, precision="fp64", batch=2)
    asm = fem.assemble(w.model)
    y, _ = fom.sweep(asm, freqs, fem.load_matrix(w.model, w.loads, w.n_rhs),
                     fem.receiver_dofs(w.model, w.receivers), method="dense")
    assert (_per_freq_rel(res.p.cpu().numpy(), y) <= _fp64_bound(_dense_kappa(asm, freqs))).all()


@pytest.mark.parametrize("ncols", [None, 1, 3, 8, 13])
def test_residual_kernel_matches_sparse_product(ncols):
    """The CSR residual against scipy's sparse product; the column counts cover every
    power-of-two column slice of the kernel (13 = 8 + 4 + 1, 3 = 2 + 1)."""
    torch = need_cuda()
    w = W.small_model(floor=True)
    api, model, F, rcv = _setup(w)
    asm = fem.assemble(w.model)
    rng = np.random.default_rng(11)
    if ncols is not None:
        Fh = rng.standard_normal((asm.n, ncols)) + 1j * rng.standard_normal((asm.n, ncols))
        F = torch.tensor(Fh, device="cuda")
    nc = F.shape[1]
    freqs = [40.0, 90.0, 333.0]
    X = rng.standard_normal((3, asm.n, nc)) + 1j * rng.standard_normal((3, asm.n, nc))
    R = api.fsi_residual(model, freqs, torch.tensor(X, device="cuda"), F).cpu().numpy()
    Fh = F.cpu().numpy()
    for i, f in enumerate(freqs):
        ref = Fh - asm.A(2 * np.pi * f) @ X[i]
        for c in range(nc):
            assert rel(R[i][:, c], ref[:, c]) <= 1e-13


@pytest.mark.parametrize("precision", ["fp32_ir", "bf16x6_ir"])
def test_cfg2_full_size_sampled_frequencies(precision):
    """Config 2 (81,792 DoF, b = 852, 96 slabs, floor impedance, 4 loads) in the launch
    configuration the benchmark times, checked at sampled frequencies against the
    oracle's block-banded GEPP."""
    w = W.config2()
    api, model, F, rcv = _setup(w)
    freqs = np.array([20.0, 233.0, 500.0])
    # cond ~ 5e7 at 20 Hz: a 1e-10 residual keeps the forward error far inside 0.1 dB.  There
    # the FP64 residual of any solution stalls near 2e-10 (the rounding floor of evaluating it),
    # which the refinement accepts as converged.
    # at 20 Hz the tensor-core factor needs about 100 GMRES steps (the FP32 one about 40)
    res = api.frf_sweep_full(model, freqs, F, rcv, precision=precision, batch=3, max_refine=160, tol=1e-10)
    print("cfg2 iterations", res.iters.tolist(), "relres", res.relres.tolist())
    # (at 20 Hz the accepted rounding floor of the scaled residual is ~1e-9)
    assert res.stats.n_unconverged == 0 and res.relres.max() <= 5e-9
    asm = fem.assemble(w.model)
    y, _ = fom.sweep(asm, freqs, fem.load_matrix(w.model, w.loads, w.n_rhs),
                     fem.receiver_dofs(w.model, w.receivers), method="banded")
    p = res.p.cpu().numpy()
    assert _per_freq_rel(p, y).max() <= 1e-6
    assert db_err(p, y) <= 0.1


@pytest.mark.parametrize("cfg", [2, 4])
def test_full_size_reciprocity(cfg):
    """At the full sizes of configs 2 and 4 (81,792 and 223,360 DoF), a property that holds
    at any size: the pressure at an interior node b per unit normal force at a shell node a
    equals rho w^2 times the shell displacement at a per unit fluid source at b (the
    coupled matrix is complex symmetric after the fluid-row scaling)."""
    torch = need_cuda()
    from paper_2310_04734_gb300 import api
    w = W.CONFIGS[cfg]()
    spec = w.model
    num = fem.Numbering(spec)
    a = num.s(3, spec.nz // 2, 0)
    b = num.p(spec.nx // 2, spec.ny // 3, spec.nz // 3)
    model = api.fsi_assemble(spec)
    n = int(model.dims.n)
    F = torch.zeros((n, 2), dtype=torch.complex128, device="cuda")
    F[a, 0] = 1.0
    F[b, 1] = 1.0
    rcv = torch.tensor([b, a], dtype=torch.int32, device="cuda")
    freqs = np.array([37.0, 211.0])
    res = api.frf_sweep_full(model, freqs, F, rcv, precision="fp32_ir", batch=2, max_refine=80, tol=1e-12)
    p = res.p.cpu().numpy()
    om = 2 * np.pi * freqs
    H_pF, H_wQ = p[:, 0, 0], p[:, 1, 1]
    gap = np.abs(H_pF - spec.rho * om ** 2 * H_wQ) / np.abs(H_pF)
    print("cfg%d reciprocity gap" % cfg, gap.tolist(), "relres", res.relres.tolist())
    assert res.stats.n_unconverged == 0 and gap.max() <= 1e-7


def _kappa1_banded(asm, freq):
    """1-norm condition estimate of the scaled system (Hager / Higham's estimator through the
    oracle's block-banded factor), for sizes where a dense condition number is out of reach.
    The scaled system is complex symmetric (reciprocity scaling of the fluid rows), so the
    adjoint solve is conj(A_s^-1 conj(v))."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla
    om = 2 * np.pi * freq
    r, c = fom.equilibrate(asm, om)
    As = (sp.diags(r) @ asm.A(om) @ sp.diags(c)).tocsc()
    lu = fom.BlockBandedLU(asm, om)
    n = asm.n
    # A_s^-1 = C^-1 A^-1 R^-1
    def inv_s(v):
        return lu.solve(np.asarray(v).ravel() / r) / c

    inv = spla.LinearOperator((n, n), dtype=complex, matvec=inv_s, rmatvec=lambda v: np.conj(inv_s(np.conj(v))))
    est = spla.onenormest(inv)
    return float(abs(As).sum(axis=0).max() * est)


@pytest.mark.slow
def test_cfg2_fp64_path_vs_oracle_banded():
    """Config 2 (81,792 DoF), plain FP64 factor and solve (the metric's denominator path)
    against the oracle's block-banded GEPP at 20, 233 and 500 Hz, bounded by
    max(1e-10, 10 kappa u) with kappa the 1-norm condition estimate of the scaled system."""
    w = W.config2()
    api, model, F, rcv = _setup(w)
    freqs = np.array([20.0, 233.0, 500.0])
    res = api.frf_sweep_full(model, freqs, F, rcv, precision="fp64", batch=3, max_refine=2, tol=1e-15,
                             allow_noconv=True)
    asm = fem.assemble(w.model)
    y, _ = fom.sweep(asm, freqs, fem.load_matrix(w.model, w.loads, w.n_rhs),
                     fem.receiver_dofs(w.model, w.receivers), method="banded")
    e = _per_freq_rel(res.p.cpu().numpy(), y)
    kap = np.array([_kappa1_banded(asm, f) for f in freqs])
    print("cfg2 fp64 vs oracle:", e.tolist(), "kappa1", kap.tolist())
    assert (e <= _fp64_bound(kap)).all()


@pytest.mark.slow
def test_cfg4_full_order_vs_oracle_banded():
    """Config 4 (223,360 DoF, b = 1396, 160 slabs, per-layer loss factors): the benchmark's
    mixed path (FP32 factor + FP64 GMRES to 1e-10) against the oracle's block-banded GEPP at
    two seeded check frequencies, <= 1e-6 relative and <= 0.1 dB."""
    w = W.config4()
    api, model, F, rcv = _setup(w)
    freqs = np.sort(w.check_freqs_hz)[[7, 31]]
    res = api.frf_sweep_full(model, freqs, F, rcv, precision="fp32_ir", batch=2, max_refine=80, tol=1e-10)
    assert res.stats.n_unconverged == 0
    asm = fem.assemble(w.model)
    y, _ = fom.sweep(asm, freqs, fem.load_matrix(w.model, w.loads, w.n_rhs),
                     fem.receiver_dofs(w.model, w.receivers), method="banded")
    p = res.p.cpu().numpy()
    print("cfg4 at", freqs.tolist(), "rel err", _per_freq_rel(p, y).tolist(), "iters", res.iters.tolist())
    assert _per_freq_rel(p, y).max() <= 1e-6
    assert db_err(p, y) <= 0.1
