"""Persistent multi-model reduced sweep (uneven reduced orders in one launch) against
the oracle's reduced sweep (dense GEPP, Eq. 11) on the same reduced matrices and
against the per-model FP64 reduced sweep, and its replay from a captured CUDA graph."""
import numpy as np
import pytest

import workloads as W
from gpu_util import need_cuda, rel
from oracle import rom as orom

pytestmark = pytest.mark.gpu


def _roms():
    from paper_2310_04734_gb300 import api
    import torch
    roms, freqs = [], []
    cases = [(2, True, (5, 4, 6), 31), (3, False, (4, 5, 7), 32), (4, True, (5, 5, 8), 33), (12, True, (6, 5, 9), 34)]
    for q, floor, (nx, ny, nz), cid in cases:
        w = W.small_model(nx=nx, ny=ny, nz=nz, floor=floor, n_loads=2, n_rcv=4, cfg_id=cid)
        model = api.fsi_assemble(w.model)
        F = api.dense_loads(w.model, w.loads, w.n_rhs)
        rcv = torch.tensor(api.receiver_dofs(w.model, w.receivers), device="cuda")
        V = api.rom_build(model, [60.0, 150.0, 250.0], q, F, kmax=128, precision="fp64", max_refine=4, tol=1e-13)
        roms.append(api.rom_project(model, V, F, rcv))
        freqs.append(np.linspace(35.0, 290.0, 11 + 3 * q))
    return roms, freqs


def test_multi_sweep_matches_per_model_sweeps():
    torch = need_cuda()
    from paper_2310_04734_gb300 import api
    roms, freqs = _roms()
    assert len({r.k for r in roms}) == len(roms) and max(r.k for r in roms) > 64
    ms = api.MultiSweep(roms, freqs)
    ms.launch()
    torch.cuda.synchronize()
    st = ms.status.cpu().numpy()
    assert set(np.unique(st)) <= {0, 3}
    # items the FP32 factor cannot refine are flagged and re-solved in FP64
    flagged = [st[o:o2] == 3 for o, o2 in zip(ms.offsets.cpu().numpy()[:-1], ms.offsets.cpu().numpy()[1:])]
    flagged = {i: flagged[slot] for slot, i in enumerate(ms.order)}
    nfix = ms.fixup(roms, freqs)
    assert nfix == int((st == 3).sum())
    u = np.finfo(np.float64).eps / 2
    for m_i, (rm, f, p, spl) in enumerate(zip(roms, freqs, ms.p, ms.spl)):
        pref, splref = api.rom_sweep(rm, f, batch=16)
        pg, pr = p.cpu().numpy(), pref.cpu().numpy()
        KR, DR, MR = (x.cpu().numpy() for x in (rm.KR, rm.DR, rm.MR))
        # the oracle's reduced sweep on the very same reduced matrices
        yo = orom.reduced_sweep(orom.ReducedModel(KR=KR, DR=DR, MR=MR, fR=rm.fR.cpu().numpy(),
                                                  CR=rm.CR.cpu().numpy()), f)
        for i, fi in enumerate(f):
            w = 2 * np.pi * fi
            A = KR + 1j * w * DR - w * w * MR
            kraw = np.linalg.cond(A, 1)   # the oracle solves the unscaled system
            assert rel(pg[i], yo[i]) <= max(1e-6, 10 * kraw * u), (rm.k, fi, rel(pg[i], yo[i]), kraw)
            A = A / np.abs(A).max(axis=1, keepdims=True)            # the row equilibration both solvers use
            kappa = np.linalg.cond(A / np.abs(A).max(axis=0, keepdims=True), 1)
            if flagged[m_i][i]:   # only systems an FP32 factor cannot refine are flagged
                assert kappa > 1e4, (rm.k, fi, kappa)
            # both are backward stable in FP64 (the multi-model kernel after refinement)
            assert rel(pg[i], pr[i]) <= max(1e-6, 10 * kappa * u), (rm.k, fi, rel(pg[i], pr[i]), kappa)
        assert np.abs(spl.cpu().numpy() - splref.cpu().numpy()).max() <= 1e-4


def test_multi_sweep_replays_from_a_cuda_graph():
    torch = need_cuda()
    from paper_2310_04734_gb300 import api
    roms, freqs = _roms()
    ms = api.MultiSweep(roms, freqs)
    ms.launch()
    torch.cuda.synchronize()
    ref = [p.clone() for p in ms.p]
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        ms.launch()   # warm-up on the capture stream
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    for p in ms.p:
        p.zero_()
    with torch.cuda.graph(g):
        ms.launch()
    for p in ms.p:
        p.zero_()
    g.replay()
    g.replay()
    torch.cuda.synchronize()
    assert all(torch.equal(a, b) for a, b in zip(ref, ms.p))
