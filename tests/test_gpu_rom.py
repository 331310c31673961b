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
