"""Benchmark: full-order frequency-response sweep of the medium coupled model.

Workload (the model the headline metric is quoted on): 1.5 x 1.5 x 6 m cavity
at 24 x 24 x 96 nodes plus the shell ring, 81,792 DoF (b = 852 per slab, 96
slabs), floor impedance, 4 seeded shell loads, 32 receivers, 481 frequencies
20..500 Hz.  A step is one batch of `--batch` frequencies through the whole
path: form A(w) -> block-banded LU stored in FP32 (the long trailing updates on
the tcgen05 tensor cores with three-plane BF16 splits, --precision bf16x6_ir;
or all on the FP32 pipe, fp32_ir) -> FP64 GMRES refinement preconditioned by the
factor, to a relative residual of 1e-10 -> receivers and SPL.  value =
frequencies / s over all ranks.  The factor store of one batch (~200 GB) is far
larger than L2, so no separate L2 flush is needed between steps.

--impl reference times the CPU oracle (oracle/, the plain FP64 restatement of
the method) on the host cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

# Relative residual of the scaled system at which refinement stops.  At 20 Hz the
# medium model's condition number is ~5e7, so 1e-8 would bound the forward error
# only by ~0.5; 1e-10 keeps it well inside 0.1 dB.
REFINE_TOL = 1e-10
METRIC = "FRF frequencies/sec at <=0.1 dB SPL error vs FP64 full-order sweep; tensor-pipe %"
UNIT = "frequencies/s"
GEMM_BYTES_PER_FLOP = 465.3e6 / 31.35e9
# DRAM bytes (read + write) per complex flop (8 M N K) of the tensor-core Schur update, from one
# ncu capture of 8 config-2 windows (585.4 + 78.3 MB for 8 x 8 x 852 x 1704 x 852 flops); the
# short-K updates move more bytes per flop, so this scaled figure is a lower bound for them
TC_BYTES_PER_FLOP = (585.4e6 + 78.3e6) / (8 * 8.0 * 852 * 1704 * 852)


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        return json.load(open(p)), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
            "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (FileNotFoundError, OSError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm = [float(r[1]) for r in self.rows if len(r) >= 9 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) >= 9 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in self.rows:
            if len(r) < 9:
                continue
            for nm, v in zip(names, r[5:9]):
                if v.strip().lower() in ("active", "1"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def run_reference(args):
    """The oracle on the host cores, timed on a bounded sample of the workload."""
    world, rank, _ = _dist()
    if rank != 0:
        return 0
    from oracle import fem, fom
    w = W.config2()
    asm = fem.assemble(w.model)
    F = fem.load_matrix(w.model, w.loads, w.n_rhs)
    rc = fem.receiver_dofs(w.model, w.receivers)
    freqs = w.freqs_hz
    sample = [freqs[(7 * i + 3) % len(freqs)] for i in range(max(1, args.warmup) + args.steps)]
    times = []
    for i, f in enumerate(sample):
        t0 = time.perf_counter()
        fom.sweep(asm, [f], F, rc, method="banded")
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(dt)
    per = sum(times) / len(times)
    cores = os.cpu_count()
    val = 1.0 / per
    line = {"metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": per * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w.name, "model_dofs": int(asm.n), "slab_block": int(asm.b), "slabs": int(asm.nz),
                       "loads": w.n_rhs, "receivers": len(w.receivers), "step": "one frequency"},
            "impl": "reference",
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{args.steps} frequencies of the 481-point grid, block-banded GEPP FP64 "
                                       f"(oracle.fom, numpy/scipy BLAS on {cores} host cores)"},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def cpu_baseline_sample(seconds_cap=40.0):
    """Oracle frequencies/s on the host cores, one config-2 frequency (bounded sample)."""
    from oracle import fem, fom
    w = W.config2()
    asm = fem.assemble(w.model)
    F = fem.load_matrix(w.model, w.loads, w.n_rhs)
    rc = fem.receiver_dofs(w.model, w.receivers)
    t0 = time.perf_counter()
    fom.sweep(asm, [233.0], F, rc, method="banded")
    dt = time.perf_counter() - t0
    return {"value": 1.0 / dt, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"1 frequency (233 Hz) of the config-2 sweep by the oracle's block-banded GEPP "
                      f"in FP64, {dt:.1f} s"}


def _sm_count(torch):
    return int(torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count)


def measure_peaks(api, kinds=("fp32_fma", "fp64_fma", "bf16_tcgen05", "tf32_tcgen05"), seconds=0.25):
    """Throughput probes of the execution units (fsi_probe_peak), TFLOP/s."""
    out = {}
    for k in kinds:
        try:
            out[k] = api.fsi_probe_peak(k, seconds)[0]
        except RuntimeError as e:   # a probe that fails leaves the derived figure in use
            out[k] = None
            print(f"peak probe {k} failed: {e}", file=sys.stderr)
    return out


def run_peaks(args):
    """Measured FP32 / FP64 FMA and tcgen05 BF16 / TF32 throughput of this GPU (one line)."""
    import torch
    from paper_2310_04734_gb300 import api
    clocks = ClockSampler(0)
    clocks.start()
    probes = measure_peaks(api, kinds=tuple(api.PEAK_KINDS), seconds=1.0)
    clk = clocks.stop()
    peaks, src = _peaks()
    print(json.dumps({"mode": "peaks", "tflops": probes, "sm_count": _sm_count(torch), "clocks": clk,
                      "measured_peaks_json": {k: peaks.get(k) for k in ("hbm_gbs", "bf16_tflops",
                                                                        "bf16_tflops_sustained")}}))
    return 0


def run_lu_window(args):
    """Batched partial LU of --batch random windows shaped like one config-2 slab step
    (2b x 3b complex, b = 852, b pivots): the factor kernels alone, a few hundred MB."""
    import torch
    from paper_2310_04734_gb300 import api
    b = 852
    m, ncols = 2 * b, 3 * b
    gen = torch.Generator(device="cuda").manual_seed(7)
    base = torch.randn((args.batch, m, ncols), dtype=torch.complex64, device="cuda", generator=gen)
    A = base.clone()
    tc = {"bf16x6_ir": "bf16x6", "bf16_ir": "bf16"}.get(args.precision, False)
    for _ in range(args.warmup):
        A.copy_(base)
        api.fsi_batched_lu(A, b, tensor_cores=tc)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    tot = 0.0
    for _ in range(args.steps):
        A.copy_(base)
        ev0.record()
        api.fsi_batched_lu(A, b, tensor_cores=tc)
        ev1.record()
        torch.cuda.synchronize()
        tot += ev0.elapsed_time(ev1)
    flops = 8.0 * args.batch * sum((m - j) * (ncols - j) for j in range(b))
    print(json.dumps({"mode": "lu_window", "precision": args.precision, "batch": args.batch,
                      "ms_per_call": tot / args.steps, "alg_tflops": flops / (tot / args.steps / 1e3) / 1e12}))
    return 0


def run_rom(args):
    """Config 4 (223,360 DoF, b = 1396, 160 slabs, 2 loads, 64 receivers): local ROM windows
    over the band (greedy expansion points with the Gram-block residual estimate, windows
    bisected while their estimate stays above tolerance), the windowed reduced sweep over
    the band's 0.5 Hz grid timed with CUDA events, and the SPL error against the full-order
    model (FP32 factor + FP64 GMRES to 1e-10) at the seeded check frequencies in the band."""
    import torch
    from paper_2310_04734_gb300 import api
    w = W.config4()
    spec = w.model
    model = api.fsi_assemble(spec)
    F = api.dense_loads(spec, w.loads, w.n_rhs)
    rcv = torch.tensor(api.receiver_dofs(spec, w.receivers), device="cuda")
    lo, hi = args.rom_band
    grid = w.freqs_hz[(w.freqs_hz >= max(lo, 1.0)) & (w.freqs_hz <= hi)]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    P = args.rom_batch_shifts
    wr = api.rom_windows(model, F, rcv, grid, q=args.rom_q, kmax=args.rom_kmax,
                         max_shifts=args.rom_max_shifts or (P if P > 1 else 12), tol=args.rom_tol,
                         max_windows=args.rom_windows, min_points=8, reuse=not args.rom_no_reuse,
                         precision=args.rom_precision, batch_shifts=P, init_points=args.rom_init_points,
                         init_windows=args.rom_init_windows)
    torch.cuda.synchronize()
    t_build = time.perf_counter() - t0
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        api.rom_windows_sweep(wr, grid, batch=256)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        p, spl = api.rom_windows_sweep(wr, grid, batch=256)
    ev1.record(stream)
    torch.cuda.synchronize()
    t_sweep = ev0.elapsed_time(ev1) / 1e3 / args.steps
    chk = w.check_freqs_hz[(w.check_freqs_hz >= grid[0]) & (w.check_freqs_hz <= grid[-1])]
    if len(chk) == 0:
        chk = grid[np.linspace(0, len(grid) - 1, 5).astype(int)]
    torch.cuda.empty_cache()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    full = api.frf_sweep_full(model, chk, F, rcv, precision="bf16x6_ir", batch=min(16, len(chk)), max_refine=80,
                              tol=1e-10, allow_noconv=True)
    torch.cuda.synchronize()
    t_full = time.perf_counter() - t0
    pr, _ = api.rom_windows_sweep(wr, chk, batch=64)
    pf = full.p.cpu().numpy()
    pm = pr.cpu().numpy()
    db = np.abs(20 * np.log10(np.abs(pm) / np.abs(pf)))
    relerr = np.abs(pm - pf) / np.abs(pf)
    print(json.dumps({
        "mode": "rom", "metric": "ROM sweep frequencies/s (config 4 band, windowed)", "value": len(grid) / t_sweep,
        "unit": UNIT, "band_hz": [float(grid[0]), float(grid[-1])], "frequencies": int(len(grid)),
        "windows": [{"lo": float(a), "hi": float(b), "k": int(k), "points": int(n), "reused_points": int(r),
                     "maxest": float(m)}
                    for a, b, k, n, r, m in zip(wr.lo, wr.hi, wr.k, wr.nshift, wr.nreused, wr.maxest)],
        "cross_window_reuse": not args.rom_no_reuse,
        "build_s": t_build, "sweep_ms": t_sweep * 1e3,
        "e2e": {"value": len(grid) / (t_build + t_sweep), "unit": UNIT, "note": "window build + one sweep"},
        "full_order_check": {"value": len(chk) / t_full, "unit": UNIT,
                             "note": "the check frequencies at full order (BF16x6 tensor-core LU + FP64 GMRES "
                                     "to 1e-10)",
                             "reduced_sweep_speedup": (len(grid) / t_sweep) / (len(chk) / t_full)},
        "check": {"frequencies": int(len(chk)), "max_spl_err_db": float(db.max()),
                  "median_spl_err_db": float(np.median(db)), "max_rel_err": float(relerr.max()),
                  "fom_unconverged": int(full.stats.n_unconverged)},
        "build": {"precision": args.rom_precision, "batch_shifts": P, "init_points": args.rom_init_points,
                  "init_windows": args.rom_init_windows, "q": args.rom_q, "kmax": args.rom_kmax, "tol": args.rom_tol},
        "dtype": "f64 reduced LU; moments by the %s factor + f64 refinement" % args.rom_precision}))
    return 0


def run_design(args):
    """Config 5's design study at reduced scale (64 seeded variants of uneven size, 101
    frequencies each): the error estimator is trained on the first 16 variants' greedy
    ROMs by the GPU training kernel; variants 0-15 get residual-driven greedy ROMs and
    16-63 estimator-driven ones; all 64 reduced sweeps run in one persistent launch
    replayed from a CUDA graph (timed); every variant is checked at 40 seeded frequencies
    by the full-order residual of its lifted reduced solutions, and frequencies above
    the residual tolerance are re-solved at full order and replaced (rom_check_resolve)."""
    import torch
    from paper_2310_04734_gb300 import api, design_study as ds
    variants = W.config5_reduced_variants(64)
    q, kmax, rounds = 6, 128, 6
    t0 = time.perf_counter()
    data = [ds.variant_samples(w, rounds, q, kmax) for w in variants[:16]]
    order = W.mlp_order(sum(len(d.T) for d in data), 2000, 256)
    st, losses = ds.train_estimator(data, W.mlp_init(), order, lr=1e-3)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    t0 = time.perf_counter()
    roms, handles, bases = [], [], []
    for i, w in enumerate(variants):
        g, h = ds.variant_rom(w, q, kmax, args.design_shifts, 1e-4, mlp_params=st.params if i >= 16 else None)
        roms.append(g.rom)
        handles.append(h)
        bases.append(g.V)
    torch.cuda.synchronize()
    t_build = time.perf_counter() - t0
    ms = api.MultiSweep(roms, [w.freqs_hz for w in variants])
    stream = torch.cuda.current_stream()
    ms.launch()
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    side.wait_stream(stream)
    with torch.cuda.stream(side):
        ms.launch()
    stream.wait_stream(side)
    torch.cuda.synchronize()
    with torch.cuda.graph(graph):
        ms.launch()
    for _ in range(args.warmup):
        graph.replay()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        graph.replay()
    ev1.record(stream)
    torch.cuda.synchronize()
    t_sweep = ev0.elapsed_time(ev1) / 1e3 / args.steps
    nfreq = sum(len(w.freqs_hz) for w in variants)
    # reduced systems the FP32 factor could not refine are re-solved in FP64 (not timed)
    nfix = ms.fixup(roms, [w.freqs_hz for w in variants])
    # checks at 40 seeded frequencies per variant: the full-order FP64 residual of the lifted
    # reduced solutions judges each one (rom_check_resolve); failures are re-solved at full
    # order and replace the reduced outputs.  The SPL error of the final outputs against the
    # full-order sweep is then measured at the same frequencies (a report, not part of the path).
    worst, worst_before, resolve, kk, resid = [], [], 0, [], []
    torch.cuda.synchronize()
    t_check = 0.0
    for i, w in enumerate(variants):
        idx = np.sort(np.random.default_rng([w.config_id, 3]).choice(len(w.freqs_hz), size=40, replace=False))
        model_i, F_i, rcv_i = handles[i]
        ti = torch.as_tensor(idx, device="cuda")
        pc, sc = ms.p[i][ti].contiguous(), ms.spl[i][ti].contiguous()
        before = pc.clone()
        t0 = time.perf_counter()
        rel, res, n = api.rom_check_resolve(model_i, bases[i], roms[i], F_i, rcv_i, w.freqs_hz[idx], pc, sc,
                                            res_tol=args.design_res_tol)
        torch.cuda.synchronize()
        t_check += time.perf_counter() - t0
        ms.p[i][ti] = pc
        ms.spl[i][ti] = sc
        resolve += n
        resid.append(float(rel.max()))
        db, pf = ds.check_variant(w, handles[i], ms.p[i], idx)
        db0 = np.abs(20.0 * np.log10(np.abs(before.cpu().numpy()) / np.abs(pf))).max(axis=(1, 2))
        worst.append(float(db.max()))
        worst_before.append(float(db0.max()))
        kk.append(int(roms[i].k))
    worst = np.array(worst)
    print(json.dumps({
        "mode": "design", "metric": "design study: reduced sweep frequencies/s (64 variants, one persistent launch)",
        "value": nfreq / t_sweep, "unit": UNIT, "variants": len(variants), "frequencies": nfreq,
        "sweep_ms": t_sweep * 1e3, "train_s": t_train, "build_s": t_build, "fp64_resolved_reduced": nfix,
        "estimator_final_loss": float(np.mean(losses[-100:])), "k": {"min": min(kk), "max": max(kk)},
        "check": {"frequencies": 40 * len(variants), "residual_tol": args.design_res_tol,
                  "resolved_full_order": resolve, "check_and_resolve_s": t_check,
                  "max_spl_err_db_before_check": float(max(worst_before)),
                  "max_spl_err_db_after_check": float(worst.max()),
                  "max_full_residual": float(max(resid)), "median_variant_max_full_residual": float(np.median(resid)),
                  "max_spl_err_db_residual_driven": float(worst[:16].max()),
                  "max_spl_err_db_estimator_driven": float(worst[16:].max()),
                  "median_worst_db_residual_driven": float(np.median(worst[:16])),
                  "median_worst_db_estimator_driven": float(np.median(worst[16:]))},
        "e2e": {"value": nfreq / (t_build + t_sweep + t_check), "unit": UNIT,
                "note": "ROM builds + one sweep + the residual check and full-order re-solves"},
        "dtype": "f32 reduced LU + f64 refinement; estimator fp16 weights / fp32 accumulation"}))
    return 0


def run_kernels(args):
    """FP64 sparse and basis kernels of the path at full size, each timed with CUDA events
    (on GB300 they are bound by the FP64 pipe rather than HBM): the CSR residual
    r = F - A(w)X (config 2, 8 frequencies x 4 loads), the Galerkin projection (config 4,
    160 columns: sparse products and V^H X), and one CGS2-orthonormalised moment build
    (config 4, one point, 24 moments per load: the basis outgrows L2 after ~36 columns)."""
    import torch
    from paper_2310_04734_gb300 import api
    out = {"mode": "kernels"}
    stream = torch.cuda.current_stream()

    def timed(fn, reps):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3 / reps

    w2 = W.config2()
    m2 = api.fsi_assemble(w2.model)
    F2 = api.dense_loads(w2.model, w2.loads, w2.n_rhs)
    n2, nnz2, nf = int(m2.dims.n), int(m2.dims.nnz), 8
    gen = torch.Generator(device="cuda").manual_seed(3)
    X = torch.randn((nf, n2, w2.n_rhs), dtype=torch.complex128, device="cuda", generator=gen)
    freqs = w2.freqs_hz[:nf]
    t = timed(lambda: api.fsi_residual(m2, freqs, X, F2), 5)
    # per frequency: CSR pattern (4 + 4/row) and values K (16), M (8), D (16) per nonzero, x gathers
    # (16 per nonzero and column, L2-served), F read and R written (16 each per row and column)
    byt = nf * (nnz2 * (4 + 16 + 8 + 16) + n2 * 4 + 2 * n2 * w2.n_rhs * 16)
    out["residual"] = {"ms": t * 1e3, "dram_model_bytes": byt, "GB_s": byt / t / 1e9, "rows": n2, "nnz": nnz2,
                       "freqs": nf, "loads": w2.n_rhs}
    del X
    w4 = W.config4()
    m4 = api.fsi_assemble(w4.model)
    F4 = api.dense_loads(w4.model, w4.loads, w4.n_rhs)
    rcv4 = torch.tensor(api.receiver_dofs(w4.model, w4.receivers), device="cuda")
    n4, k = int(m4.dims.n), 160
    # any n x k block has the projection's cost; random columns scaled to unit norm
    Q = torch.randn((n4, k), dtype=torch.complex128, device="cuda", generator=gen) / np.sqrt(2.0 * n4)
    t = timed(lambda: api.rom_project(m4, Q, F4, rcv4), 2)
    out["projection"] = {"ms": t * 1e3, "n": n4, "k": k, "fp64_tflops": 3 * 8.0 * n4 * k * k / t / 1e12}
    del Q
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    V = api.rom_build(m4, [200.0], 24, F4, kmax=64)
    torch.cuda.synchronize()
    out["rom_build"] = {"s": time.perf_counter() - t0, "workload": "config 4, one point at 200 Hz",
                        "moments_per_load": 24, "k": int(V.shape[1]),
                        "basis_bytes": int(V.shape[1]) * n4 * 16}
    print(json.dumps(out))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--batch", type=int, default=96)
    ap.add_argument("--restart", type=int, default=40, help="GMRES restart length of the refinement")
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--precision", default="bf16x6_ir", choices=["fp32_ir", "bf16x6_ir", "bf16_ir", "fp64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--fp64-sample", type=int, default=4, help="frequencies timed on the plain FP64 path")
    ap.add_argument("--rom-band", type=float, nargs=2, default=[1.0, 1000.0])
    ap.add_argument("--rom-q", type=int, default=16)
    ap.add_argument("--rom-kmax", type=int, default=400)
    ap.add_argument("--rom-tol", type=float, default=1e-4)
    ap.add_argument("--rom-windows", type=int, default=16)
    ap.add_argument("--rom-batch-shifts", type=int, default=1,
                    help="expansion points factored and solved together; with > 1 every window is built from "
                         "that many points at once (no greedy additions, failing windows are bisected)")
    ap.add_argument("--rom-init-points", type=int, default=0)
    ap.add_argument("--rom-init-windows", type=int, default=1)
    ap.add_argument("--rom-max-shifts", type=int, default=0)
    ap.add_argument("--rom-precision", default="fp32_ir", choices=["fp32_ir", "bf16x6_ir", "fp64"])
    ap.add_argument("--rom-no-reuse", action="store_true",
                    help="windows start from fresh points instead of their enclosing windows' points")
    ap.add_argument("--design-shifts", type=int, default=16)
    ap.add_argument("--design-res-tol", type=float, default=1e-6,
                    help="full-order relative residual above which a check frequency is re-solved at full order")
    ap.add_argument("--mode", default="sweep", choices=["sweep", "lu_window", "rom", "design", "kernels", "peaks"],
                    help="lu_window: only the batched band-LU of config-2-sized windows (for kernel profiling)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.mode == "lu_window":
        return run_lu_window(args)
    if args.mode == "rom":
        return run_rom(args)
    if args.mode == "design":
        return run_design(args)
    if args.mode == "kernels":
        return run_kernels(args)
    if args.mode == "peaks":
        return run_peaks(args)

    import torch
    from paper_2310_04734_gb300 import api

    world, rank, local = _dist()
    torch.cuda.set_device(local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        pg = dist

    w = W.config2()
    spec = w.model
    model = api.fsi_assemble(spec)
    F = api.dense_loads(spec, w.loads, w.n_rhs)
    rcv = torch.tensor(api.receiver_dofs(spec, w.receivers), device="cuda")
    freqs = w.freqs_hz
    B = args.batch
    nsteps = args.warmup + args.steps

    from paper_2310_04734_gb300.sharding import batch_indices

    def batch_freqs(step):
        # rank-sharded batches of the 481-point grid (wrapping); each rank sweeps its own frequencies
        return freqs[batch_indices(len(freqs), B, world, rank, step)]

    # one workspace serves the device-buffer steps and the host-buffer (e2e) steps
    ws_bytes = max(api.frf_sweep_workspace(model, args.precision, B, w.n_rhs, len(w.receivers), restart=args.restart),
                   api.frf_sweep_workspace(model, args.precision, B, w.n_rhs, len(w.receivers), host_io=True,
                                           restart=args.restart))
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    kw = dict(precision=args.precision, batch=B, max_refine=160, tol=REFINE_TOL, workspace=ws, allow_noconv=True,
              restart=args.restart)
    for s in range(args.warmup):
        api.frf_sweep_full(model, batch_freqs(s), F, rcv, **kw)
    torch.cuda.synchronize()
    if pg:
        pg.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    kern_ms = np.zeros(12)
    kern_flops = np.zeros(12)
    kern_n = np.zeros(12, dtype=np.int64)
    launches = 0
    unconv = 0
    iters = []
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("timed")
    ev0.record(stream)
    for s in range(args.warmup, nsteps):
        r = api.frf_sweep_full(model, batch_freqs(s), F, rcv, **kw)
        unconv += int(r.stats.n_unconverged)
        launches += int(r.stats.launches)
        iters.extend(r.iters.tolist())
    ev1.record(stream)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    clk = clocks.stop()
    # per-kernel times from a separate pass over the first timed batch (events around every
    # launch), so the headline comes from the un-instrumented steps
    rp = api.frf_sweep_full(model, batch_freqs(args.warmup), F, rcv, profile=True, **kw)
    kern_ms += np.array(rp.stats.kernel_ms[:])
    kern_flops += np.array(rp.stats.kernel_flops[:])
    kern_n += np.array(rp.stats.kernel_launches[:])
    prof_ms = float(sum(rp.stats.kernel_ms[:]))
    t_ms = ev0.elapsed_time(ev1)
    if pg:
        t = torch.tensor([t_ms], device="cuda", dtype=torch.float64)
        pg.all_reduce(t, op=pg.ReduceOp.MAX)
        t_ms = float(t.item())
    total_freqs = args.steps * B * world
    value = total_freqs / (t_ms / 1e3)

    # end to end: same metric through the C ABI with host buffers (pinned), copies inside the call
    e2e = None
    if not args.no_e2e:
        Fh = F.cpu().numpy()
        Fpin = torch.from_numpy(np.asfortranarray(Fh).T.copy()).pin_memory()   # column-major bytes
        Fview = Fpin.numpy().T
        rh = rcv.cpu().numpy()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ne = max(1, min(3, args.steps))
        for s in range(ne):   # the timed steps' frequencies again
            api.frf_sweep_full(model, batch_freqs(args.warmup + s), Fview, rh, host_io=True, **kw)
        torch.cuda.synchronize()
        te = time.perf_counter() - t0
        h2d = Fh.size * 16 + rh.size * 4
        d2h = B * rh.size * w.n_rhs * (16 + 8)
        e2e = {"value": ne * B * world / te, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h)}

    # plain FP64 full-order sweep on the same GPU (the metric's denominator), sampled
    fp64 = None
    if args.fp64_sample > 0:
        # seeded frequencies spread over the band (config 2's check-frequency stream)
        fs = np.sort(np.random.default_rng([2, 3]).choice(freqs, size=args.fp64_sample, replace=False))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r64 = api.frf_sweep_full(model, fs, F, rcv, precision="fp64", batch=len(fs), max_refine=1)
        torch.cuda.synchronize()
        t64 = time.perf_counter() - t0
        rmix = api.frf_sweep_full(model, fs, F, rcv, precision=args.precision, batch=len(fs), max_refine=60,
                                  tol=REFINE_TOL, allow_noconv=True)
        p64 = r64.p.cpu().numpy()
        pm = rmix.p.cpu().numpy()
        fp64 = {"value": len(fs) / t64, "unit": UNIT, "sample": f"{len(fs)} frequencies",
                "max_spl_err_db_mixed_vs_fp64": float(np.max(np.abs(20 * np.log10(np.abs(pm) / np.abs(p64))))),
                "max_rel_err_mixed_vs_fp64": float(np.max(np.abs(pm - p64) / np.abs(p64)))}

    peaks, src = _peaks()
    b, nz = int(model.dims.b), int(model.dims.nz)
    # the block LU's algorithmic count is (8/3 + 8) b^3 real flops per slab step (the LU of a b x b
    # complex block plus one b^3 complex product; the coupling blocks are sparse); the band LU with
    # pivoting across the stacked panel of two slabs executes
    # sum_j 8 (2b - j)(3b - j) = 8 (6 - 5/2 + 1/3) b^3 = 30.67 b^3, so each launch's executed
    # count is credited with the fraction alg_frac of algorithmic work
    alg_step = (8.0 / 3.0 + 8.0) * b ** 3
    exec_step = 8.0 * (6.0 - 2.5 + 1.0 / 3.0) * b ** 3
    alg_frac = alg_step / exec_step
    alg_per_freq = alg_step * (nz - 1)
    tensor = args.precision in ("bf16x6_ir", "bf16_ir")
    g = 10 if tensor else 0
    t_dom = kern_ms[g] / 1e3
    exec_rate = kern_flops[g] / t_dom / 1e12 if t_dom > 0 else None
    alg_rate = exec_rate * alg_frac if exec_rate else None
    probes = measure_peaks(api, ("fp32_fma", "bf16_tcgen05") if not tensor else ("bf16_tcgen05", "fp32_fma"))
    if tensor:
        nprod = 6 if args.precision == "bf16x6_ir" else 1
        peak = float(peaks["bf16_tflops"]) / nprod
        roofline = {"bound": "tensor",
                    "kernel": f"tc_gemm_kernel (tcgen05 kind::f16, BF16 operands, {nprod} product(s) per term, TMA-fed)",
                    "achieved": alg_rate, "peak": peak, "unit": "TFLOP/s",
                    "frac": (alg_rate / peak) if alg_rate else None,
                    "achieved_executed": exec_rate, "frac_executed": (exec_rate / peak) if exec_rate else None,
                    "tensor_pipe_frac": (exec_rate * nprod / float(peaks["bf16_tflops"])) if exec_rate else None,
                    "traffic": (TC_BYTES_PER_FLOP * kern_flops[g] / max(kern_n[g], 1)) if nprod == 6 else None,
                    "traffic_unit": "bytes per launch (mean launch; scaled from an ncu capture of the Schur update, "
                                    "a lower bound for the short-K launches)",
                    "peak_source": f"of measured: bf16 {peaks['bf16_tflops']} TFLOP/s (MEASURED_PEAKS.json) / "
                                   f"{nprod} product(s); probe of this run {probes.get('bf16_tcgen05')}"}
    else:
        # DRAM bytes per executed flop of the trailing update, from an ncu capture (C read-modify-write)
        traffic = GEMM_BYTES_PER_FLOP * kern_flops[g] / max(kern_n[g], 1)
        sm_max = float(peaks.get("sm_max_mhz", 2070.0))
        derived = _sm_count(torch) * 128 * 2 * sm_max * 1e6 / 1e12
        peak = probes.get("fp32_fma") or derived
        roofline = {"bound": "alu", "kernel": "cgemm_f32_kernel (complex GEMM updates of the band LU, FP32 SIMT)",
                    "achieved": alg_rate, "peak": peak, "unit": "TFLOP/s",
                    "frac": (alg_rate / peak) if alg_rate else None,
                    "achieved_executed": exec_rate, "frac_executed": (exec_rate / peak) if exec_rate else None,
                    "traffic": traffic,
                    "traffic_unit": "bytes per launch (mean launch; scaled from an ncu capture)",
                    "peak_source": "of measured: FP32 FMA probe of this run (fsi_probe_peak)" if probes.get("fp32_fma")
                                   else f"derived: {_sm_count(torch)} SM x 128 FP32 lanes x 2 x {sm_max:.0f} MHz",
                    "peak_derived": derived}
    roofline.update({
        "kernel_share_of_profiled": float(kern_ms[g] / max(prof_ms, 1e-9)),
        "alg_flops_note": "achieved = executed flops x %.4f: the block LU's algorithmic work is 10.67 b^3 per slab step, the band LU "
                          "executes 30.67 b^3 (pivoting across the stacked panel makes the coupling blocks dense)"
                          % alg_frac,
        "lu_alg_tflops_end_to_end": alg_per_freq * value / 1e12,
        "measured_probes_tflops": probes})
    shares = {k: {"ms": float(kern_ms[i]), "launches": int(kern_n[i]),
                  "share": float(kern_ms[i] / max(kern_ms.sum(), 1e-9))}
              for i, k in enumerate(["gemm", "panel", "trsm", "laswp", "form", "shift", "solve_tri", "resid",
                                         "solve_gemv", "pack", "tcgemm"])}

    if rank == 0:
        cpu = None
        if world == 1 and not args.no_cpu_baseline:
            cpu = cpu_baseline_sample()
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": t_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": {"fp32_ir": "f32 factor + f64 refinement",
                          "bf16x6_ir": "f32 factor (tensor-core BF16x6 updates) + f64 refinement",
                          "bf16_ir": "bf16 tensor-core updates, f32 factor storage + f64 refinement",
                          "fp64": "f64"}[args.precision],
                "data": "synthetic",
                "config": {"workload": w.name, "model_dofs": int(model.dims.n), "slab_block": int(model.dims.b),
                           "slabs": int(model.dims.nz), "loads": w.n_rhs, "receivers": len(w.receivers),
                           "batch_frequencies": B, "refine_tol": REFINE_TOL, "parallelism": f"replicas{world}",
                           "l2": f"inputs larger than L2 (factor store ~{2.2 * B:.0f} GB per batch)"},
                "roofline": roofline, "kernels": shares, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": launches, "clocks": clk, "fp64_full_order": fp64,
                "refine_iters": {"max": int(max(iters)), "mean": float(np.mean(iters)), "unconverged": unconv,
                                 "method": "GMRES(%d) on the FP64 system, preconditioned by the band LU (%s)"
                                           % (args.restart, args.precision)},
                "peaks_source": src}
        print(json.dumps(line), flush=True)
    if pg:
        pg.barrier()
        pg.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
