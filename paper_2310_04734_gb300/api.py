"""Python binding of the C ABI (include/fsi.h): argument marshalling only.

Every step of the computation runs in libfsi.so's CUDA kernels.  PyTorch is
used for device memory (caller-owned buffers) and the current CUDA stream.
Function names follow the C entry points.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass
from typing import Optional, Sequence

import numpy as np

from . import _lib as L

FSI_FP64 = 0
FSI_FP32_IR = 1
FSI_BF16X6_IR = 2
FSI_BF16_IR = 3
PRECISIONS = {"fp64": FSI_FP64, "fp32_ir": FSI_FP32_IR, "bf16x6_ir": FSI_BF16X6_IR, "bf16_ir": FSI_BF16_IR}


def _torch():
    import torch
    return torch


def _stream_ptr(stream=None) -> C.c_void_p:
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _ptr(t) -> C.c_void_p:
    return C.c_void_p(t.data_ptr())


def _desc(spec):
    """Marshal a workloads.ModelSpec into fsi_model_desc (keeps the eta array alive)."""
    eta = np.ascontiguousarray(np.asarray(spec.eta, dtype=np.float64))
    d = L.fsi_model_desc()
    d.Lx, d.Ly, d.Lz = spec.Lx, spec.Ly, spec.Lz
    d.nx, d.ny, d.nz = spec.nx, spec.ny, spec.nz
    d.c, d.rho = spec.c, spec.rho
    d.E, d.nu, d.rho_s, d.t = spec.E, spec.nu, spec.rho_s, spec.t
    d.eta = eta.ctypes.data_as(L.c_double_p)
    d.n_eta = int(eta.size)
    if spec.Z_floor is not None:
        d.has_floor = 1
        d.Z_re, d.Z_im = float(np.real(spec.Z_floor)), float(np.imag(spec.Z_floor))
    return d, eta


def fsi_model_dims(spec) -> L.fsi_dims:
    lib = L.load()
    d, keep = _desc(spec)
    out = L.fsi_dims()
    L.check(lib.fsi_model_dims(C.byref(d), C.byref(out)), "fsi_model_dims")
    return out


def fsi_assemble_host(spec):
    """Host CSR (rowptr, col, K, M, D) assembled by the library's C++ code."""
    lib = L.load()
    dims = fsi_model_dims(spec)
    d, keep = _desc(spec)
    rowptr = np.empty(dims.n + 1, np.int32)
    col = np.empty(dims.nnz, np.int32)
    K = np.empty(dims.nnz, np.complex128)
    M = np.empty(dims.nnz, np.float64)
    D = np.empty(dims.nnz, np.complex128)
    L.check(lib.fsi_assemble_host(C.byref(d), rowptr.ctypes.data_as(L.c_int32_p),
                                  col.ctypes.data_as(L.c_int32_p), C.c_void_p(K.ctypes.data),
                                  M.ctypes.data_as(L.c_double_p), C.c_void_p(D.ctypes.data)),
            "fsi_assemble_host")
    return dims, rowptr, col, K, M, D


@dataclass
class DeviceModel:
    spec: object
    dims: L.fsi_dims
    buf: object   # torch uint8 tensor on the device


def fsi_assemble(spec, device="cuda") -> DeviceModel:
    """Assemble on the host and upload into a torch-allocated device buffer."""
    torch = _torch()
    lib = L.load()
    dims = fsi_model_dims(spec)
    buf = torch.empty(int(dims.model_bytes) + 256, dtype=torch.uint8, device=device)
    off = (-buf.data_ptr()) % 256
    view = buf[off:off + int(dims.model_bytes)]
    d, keep = _desc(spec)
    L.check(lib.fsi_assemble(C.byref(d), _ptr(view), C.c_size_t(int(dims.model_bytes)), _stream_ptr()),
            "fsi_assemble")
    return DeviceModel(spec=spec, dims=dims, buf=view)


REFINE = {"ir": 0, "gmres": 1}


def _opts(precision, batch, max_refine, tol, host_io, profile=False, refine="gmres",
          restart=20) -> L.fsi_solve_opts:
    o = L.fsi_solve_opts()
    o.profile = int(bool(profile))
    o.refine = REFINE[refine] if isinstance(refine, str) else int(refine)
    o.restart = int(restart)
    o.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    o.batch = int(batch)
    o.max_refine = int(max_refine)
    o.tol = float(tol)
    o.host_io = int(bool(host_io))
    return o


def frf_sweep_workspace(model: DeviceModel, precision="fp32_ir", batch=8, nrhs=1, nrcv=1,
                        host_io=False, refine="gmres", restart=20) -> int:
    lib = L.load()
    o = _opts(precision, batch, 1, 1e-8, host_io, refine=refine, restart=restart)
    nb = C.c_size_t()
    L.check(lib.frf_sweep_workspace(C.byref(model.dims), C.byref(o), nrhs, nrcv, C.byref(nb)),
            "frf_sweep_workspace")
    return nb.value


@dataclass
class SweepResult:
    p: object          # [nf][nrcv][nrhs] complex128 (torch on device, or numpy with host_io)
    spl: object
    iters: np.ndarray
    relres: np.ndarray
    stats: L.fsi_sweep_stats


def frf_sweep_full(model: DeviceModel, freqs_hz: Sequence[float], F, rcv, precision="fp32_ir",
                   batch=8, max_refine=10, tol=1e-8, host_io=False, workspace=None,
                   allow_noconv=False, profile=False, refine=None, restart=20) -> SweepResult:
    """Full-order sweep.  F: n x nrhs complex128 (torch CUDA tensor, or numpy with host_io);
    rcv: receiver DoF indices (torch int32 CUDA tensor, or numpy with host_io)."""
    torch = _torch()
    lib = L.load()
    f = np.ascontiguousarray(np.asarray(freqs_hz, dtype=np.float64))
    nf = int(f.size)
    if host_io:
        Fh = np.asfortranarray(np.asarray(F, dtype=np.complex128))
        nrhs = Fh.shape[1] if Fh.ndim == 2 else 1
        Fbuf = Fh
        Fp = C.c_void_p(Fh.ctypes.data)
        rh = np.ascontiguousarray(np.asarray(rcv, dtype=np.int32))
        nrcv = int(rh.size)
        rp = C.c_void_p(rh.ctypes.data)
        p = np.empty((nf, nrcv, nrhs), np.complex128)
        spl = np.empty((nf, nrcv, nrhs), np.float64)
        pp, sp = C.c_void_p(p.ctypes.data), C.c_void_p(spl.ctypes.data)
    else:
        nrhs = F.shape[1] if F.dim() == 2 else 1
        Fbuf = F.t().contiguous() if F.dim() == 2 else F.contiguous()   # column-major n x nrhs
        Fp = _ptr(Fbuf)
        rbuf = rcv.to(torch.int32).contiguous()
        nrcv = int(rbuf.numel())
        rp = _ptr(rbuf)
        p = torch.empty((nf, nrcv, nrhs), dtype=torch.complex128, device=F.device)
        spl = torch.empty((nf, nrcv, nrhs), dtype=torch.float64, device=F.device)
        pp, sp = _ptr(p), _ptr(spl)
    if refine is None:
        refine = "ir" if precision == "fp64" else "gmres"
    o = _opts(precision, min(batch, nf), max_refine, tol, host_io, profile, refine, restart)
    need = C.c_size_t()
    L.check(lib.frf_sweep_workspace(C.byref(model.dims), C.byref(o), nrhs, nrcv, C.byref(need)),
            "frf_sweep_workspace")
    ws = workspace
    if ws is None or ws.numel() < need.value:
        ws = torch.empty(need.value, dtype=torch.uint8, device="cuda")
    iters = np.zeros(nf, np.int32)
    relres = np.zeros(nf, np.float64)
    stats = L.fsi_sweep_stats()
    st = lib.frf_sweep_full(C.byref(model.dims), _ptr(model.buf), f.ctypes.data_as(L.c_double_p), nf, Fp,
                            nrhs, rp, nrcv, C.byref(o), _ptr(ws), C.c_size_t(ws.numel()), pp, sp,
                            iters.ctypes.data_as(L.c_int32_p), relres.ctypes.data_as(L.c_double_p),
                            C.byref(stats), _stream_ptr())
    if not (allow_noconv and st == -5):
        L.check(st, "frf_sweep_full")
    return SweepResult(p=p, spl=spl, iters=iters, relres=relres, stats=stats)


def fsi_residual(model: DeviceModel, freqs_hz, X, F):
    """R_f = F - A(w_f) X_f (unscaled FP64).  X: [nf][n][nrhs] torch complex128, F: [n][nrhs]."""
    torch = _torch()
    lib = L.load()
    f = np.ascontiguousarray(np.asarray(freqs_hz, dtype=np.float64))
    nf = int(f.size)
    Xc = X.transpose(1, 2).contiguous()          # [nf][nrhs][n]
    Fc = F.t().contiguous()
    R = torch.empty_like(Xc)
    L.check(lib.fsi_residual(C.byref(model.dims), _ptr(model.buf), f.ctypes.data_as(L.c_double_p), nf,
                             _ptr(Xc), _ptr(Fc), int(F.shape[1]), _ptr(R), _stream_ptr()), "fsi_residual")
    return R.transpose(1, 2)


def fsi_batched_lu(A, npiv: int, tensor_cores=False):
    """In-place batched partial LU of row-major A [batch][m][ncols] (complex64 or complex128 CUDA);
    complex64 with tensor_cores=True (or "bf16x6") runs the long trailing updates on tcgen05 with
    three-plane BF16 splits (FP32-level), tensor_cores="bf16" with one plane (plain BF16)."""
    torch = _torch()
    lib = L.load()
    assert A.is_contiguous() and A.dim() == 3
    batch, m, ncols = A.shape
    if A.dtype == torch.complex128:
        prec = FSI_FP64
    elif not tensor_cores:
        prec = FSI_FP32_IR
    else:
        prec = FSI_BF16_IR if tensor_cores == "bf16" else FSI_BF16X6_IR
    ipiv = torch.empty((batch, npiv), dtype=torch.int32, device=A.device)
    need = C.c_size_t()
    L.check(lib.fsi_lu_workspace(prec, batch, m, ncols, npiv, C.byref(need)), "fsi_lu_workspace")
    ws = torch.empty(need.value, dtype=torch.uint8, device=A.device)
    nsing = C.c_int(0)
    L.check(lib.fsi_batched_lu(prec, batch, m, ncols, npiv, _ptr(A), ncols, m * ncols, _ptr(ipiv), _ptr(ws),
                               C.c_size_t(need.value), C.byref(nsing), _stream_ptr()), "fsi_batched_lu")
    return ipiv, nsing.value


def fsi_set_wait_limit(spins: int = 0):
    """Spin limit of the tensor-core kernels' bounded waits (0: the default)."""
    L.check(L.load().fsi_set_wait_limit(int(spins)), "fsi_set_wait_limit")


PEAK_KINDS = {"fp32_fma": 0, "fp64_fma": 1, "bf16_tcgen05": 2, "tf32_tcgen05": 3, "bf16_tcgen05_n128": 4}


def fsi_probe_peak(kind: str, seconds: float = 0.2):
    """Measured throughput (TFLOP/s, kernel ms) of one execution unit (see PEAK_KINDS)."""
    torch = _torch()
    scratch = torch.zeros(1024, dtype=torch.uint8, device="cuda")
    tf, ms = C.c_double(0.0), C.c_double(0.0)
    L.check(L.load().fsi_probe_peak(PEAK_KINDS[kind], float(seconds), _ptr(scratch), C.byref(tf), C.byref(ms),
                                    _stream_ptr()), "fsi_probe_peak")
    return tf.value, ms.value


def fsi_batched_lu_noalloc(A, npiv: int):
    """Same as fsi_batched_lu, through the entry point that allocates nothing.

    For callers that cannot allocate device memory: no workspace is created
    here or in the library; the kernels' status flags live in a fixed device
    array inside libfsi.so (at most 4095 matrices per call).  Calls that overlap
    on the GPU share that array and must not run concurrently.
    """
    lib = L.load()
    assert A.is_contiguous() and A.dim() == 3
    torch = _torch()
    batch, m, ncols = A.shape
    prec = FSI_FP64 if A.dtype == torch.complex128 else FSI_FP32_IR
    ipiv = torch.empty((batch, npiv), dtype=torch.int32, device=A.device)
    nsing = C.c_int(0)
    L.check(lib.fsi_batched_lu_noalloc(prec, batch, m, ncols, npiv, _ptr(A), ncols, m * ncols, _ptr(ipiv),
                                       C.byref(nsing), _stream_ptr()), "fsi_batched_lu_noalloc")
    return ipiv, nsing.value


def _rom_opts(precision="fp32_ir", max_refine=10, tol=1e-10, second_order=-1, batch_shifts=1):
    o = L.fsi_rom_opts()
    o.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    o.max_refine = int(max_refine)
    o.tol = float(tol)
    o.second_order = int(second_order)
    o.batch_shifts = int(batch_shifts)
    return o


def rom_build(model: DeviceModel, shifts_hz, q: int, F, kmax: int, precision="fp32_ir", max_refine=10,
              tol=1e-10, second_order=-1, batch_shifts=1):
    """Rational Arnoldi basis V (n x k complex128, column-major as a [k][n] tensor transposed);
    batch_shifts expansion points are factored and their first-order moments solved together."""
    torch = _torch()
    lib = L.load()
    s = np.ascontiguousarray(np.asarray(shifts_hz, dtype=np.float64))
    nrhs = F.shape[1]
    o = _rom_opts(precision, max_refine, tol, second_order, batch_shifts)
    need = C.c_size_t()
    L.check(lib.rom_workspace(C.byref(model.dims), nrhs, q, kmax, C.byref(o), C.byref(need)), "rom_workspace")
    ws = torch.empty(need.value, dtype=torch.uint8, device="cuda")
    Fc = F.t().contiguous()
    Vt = torch.zeros((kmax, model.dims.n), dtype=torch.complex128, device="cuda")
    k = C.c_int(0)
    L.check(lib.rom_build(C.byref(model.dims), _ptr(model.buf), s.ctypes.data_as(L.c_double_p), int(s.size), q,
                          _ptr(Fc), nrhs, kmax, C.byref(o), _ptr(ws), C.c_size_t(need.value), _ptr(Vt),
                          C.byref(k), _stream_ptr()), "rom_build")
    return Vt[:k.value].t()


@dataclass
class DeviceROM:
    KR: object
    DR: object
    MR: object
    fR: object
    CR: object

    @property
    def k(self) -> int:
        return int(self.KR.shape[0])


def rom_project(model: DeviceModel, V, F, rcv) -> DeviceROM:
    """Galerkin projection; V: n x k (torch, any layout), F: n x nrhs, rcv: int tensor."""
    torch = _torch()
    lib = L.load()
    n, k = V.shape
    nrhs = F.shape[1]
    Vc = V.t().contiguous()          # column-major n x k
    Fc = F.t().contiguous()
    r = rcv.to(torch.int32).contiguous()
    nrcv = int(r.numel())
    ws = torch.empty(max(n * k * 16, 1) + 3 * 16 * k * k * 64, dtype=torch.uint8, device="cuda")
    KR = torch.empty((k, k), dtype=torch.complex128, device="cuda")
    DR = torch.empty_like(KR)
    MR = torch.empty_like(KR)
    fR = torch.empty((nrhs, k), dtype=torch.complex128, device="cuda")
    CR = torch.empty((k, nrcv), dtype=torch.complex128, device="cuda")
    L.check(lib.rom_project(C.byref(model.dims), _ptr(model.buf), _ptr(Vc), k, _ptr(Fc), nrhs, _ptr(r), nrcv,
                            _ptr(ws), C.c_size_t(ws.numel()), _ptr(KR), _ptr(DR), _ptr(MR), _ptr(fR), _ptr(CR),
                            _stream_ptr()), "rom_project")
    # buffers are column-major: transpose views give the row-major matrices
    return DeviceROM(KR=KR.t(), DR=DR.t(), MR=MR.t(), fR=fR.t(), CR=CR.t())


def rom_sweep(rom: DeviceROM, freqs_hz, batch: int = 256, precision: str = "fp64", return_fp64: bool = False):
    """Reduced sweep: receiver pressures [nf][nrcv][nrhs] and SPL (torch, device).  precision
    "fp32_ir" (k <= 128) refines FP32 LUs against the FP64 residual; with return_fp64 the
    per-frequency flags of FP64 re-solves are returned as well."""
    torch = _torch()
    lib = L.load()
    f = np.ascontiguousarray(np.asarray(freqs_hz, dtype=np.float64))
    nf = int(f.size)
    k = rom.k
    nrhs = rom.fR.shape[1]
    nrcv = rom.CR.shape[0]
    cm = lambda X: X.t().contiguous()   # column-major buffers
    KR, DR, MR, fR, CR = cm(rom.KR), cm(rom.DR), cm(rom.MR), cm(rom.fR), cm(rom.CR)
    bt = min(batch, nf)
    prec = PRECISIONS[precision]
    need = C.c_size_t()
    L.check(lib.rom_sweep_workspace(k, nrhs, nrcv, bt, prec, C.byref(need)), "rom_sweep_workspace")
    ws = torch.empty(need.value, dtype=torch.uint8, device="cuda")
    p = torch.empty((nf, nrcv, nrhs), dtype=torch.complex128, device="cuda")
    spl = torch.empty((nf, nrcv, nrhs), dtype=torch.float64, device="cuda")
    fb = np.zeros(nf, np.int32)
    L.check(lib.rom_sweep(k, _ptr(KR), _ptr(DR), _ptr(MR), _ptr(fR), _ptr(CR), nrhs, nrcv,
                          f.ctypes.data_as(L.c_double_p), nf, bt, prec, _ptr(ws), C.c_size_t(need.value), _ptr(p),
                          _ptr(spl), fb.ctypes.data_as(L.c_int32_p), _stream_ptr()), "rom_sweep")
    if return_fp64:
        return p, spl, fb
    return p, spl


def rom_residual_check(model: DeviceModel, V, rom: DeviceROM, F, freqs_hz, batch: int = 16) -> np.ndarray:
    """Full-order FP64 residual |f - A(w) V x_R| / |f| of the reduced solutions at the given
    frequencies, per load column ([nf][nrhs] host array). V: the n x k basis rom was projected with."""
    torch = _torch()
    lib = L.load()
    f = np.ascontiguousarray(np.asarray(freqs_hz, dtype=np.float64))
    nf = int(f.size)
    k = rom.k
    nrhs = int(F.shape[1])
    cm = lambda X: X.t().contiguous()
    KR, DR, MR, fR = cm(rom.KR), cm(rom.DR), cm(rom.MR), cm(rom.fR)
    Vc, Fc = cm(V), cm(F)
    bt = min(batch, nf)
    need = C.c_size_t()
    L.check(lib.rom_residual_check_workspace(C.byref(model.dims), k, nrhs, bt, C.byref(need)),
            "rom_residual_check_workspace")
    ws = torch.empty(need.value, dtype=torch.uint8, device="cuda")
    out = np.empty((nf, nrhs), np.float64)
    L.check(lib.rom_residual_check(C.byref(model.dims), _ptr(model.buf), _ptr(Vc), k, _ptr(KR), _ptr(DR), _ptr(MR),
                                   _ptr(fR), _ptr(Fc), nrhs, f.ctypes.data_as(L.c_double_p), nf, bt, _ptr(ws),
                                   C.c_size_t(need.value), out.ctypes.data_as(L.c_double_p), _stream_ptr()),
            "rom_residual_check")
    return out


def rom_check_resolve(model: DeviceModel, V, rom: DeviceROM, F, rcv, freqs_hz, p, spl, res_tol: float,
                      precision="fp32_ir", batch: int = 8, max_refine: int = 60, tol: float = 1e-10):
    """Judge the reduced outputs p / spl ([nf][nrcv][nrhs] torch, device, updated in place) by the
    full-order FP64 residual of the lifted reduced solutions; frequencies above res_tol are solved
    again at full order and their outputs replace the reduced ones.  Returns (relres [nf][nrhs],
    resolved [nf] 0/1, count)."""
    torch = _torch()
    lib = L.load()
    f = np.ascontiguousarray(np.asarray(freqs_hz, dtype=np.float64))
    nf = int(f.size)
    k = rom.k
    nrhs = int(F.shape[1])
    cm = lambda X: X.t().contiguous()
    KR, DR, MR, fR = cm(rom.KR), cm(rom.DR), cm(rom.MR), cm(rom.fR)
    Vc, Fc = cm(V), cm(F)
    r = rcv.to(torch.int32).contiguous()
    nrcv = int(r.numel())
    assert p.is_contiguous() and spl.is_contiguous() and p.shape == (nf, nrcv, nrhs)
    bt = min(batch, nf)
    o = _opts(precision, bt, max_refine, tol, False, refine="ir" if precision == "fp64" else "gmres")
    need = C.c_size_t()
    L.check(lib.rom_check_resolve_workspace(C.byref(model.dims), k, nrhs, nrcv, bt, C.byref(o), C.byref(need)),
            "rom_check_resolve_workspace")
    ws = torch.empty(need.value, dtype=torch.uint8, device="cuda")
    rel = np.empty((nf, nrhs), np.float64)
    res = np.zeros(nf, np.int32)
    cnt = C.c_int(0)
    L.check(lib.rom_check_resolve(C.byref(model.dims), _ptr(model.buf), _ptr(Vc), k, _ptr(KR), _ptr(DR), _ptr(MR),
                                  _ptr(fR), _ptr(Fc), nrhs, _ptr(r), nrcv, f.ctypes.data_as(L.c_double_p), nf, bt,
                                  float(res_tol), C.byref(o), _ptr(ws), C.c_size_t(need.value), _ptr(p), _ptr(spl),
                                  rel.ctypes.data_as(L.c_double_p), res.ctypes.data_as(L.c_int32_p), C.byref(cnt),
                                  _stream_ptr()), "rom_check_resolve")
    return rel, res, cnt.value


def rom_save(path: str, rom: DeviceROM, shifts_hz=(), V=None, band=(0.0, 0.0)):
    """Write one reduced model (with its expansion points and, optionally, its basis V) to path."""
    lib = L.load()
    k = rom.k
    cm = lambda X: X.t().contiguous()
    bufs = [cm(rom.KR), cm(rom.DR), cm(rom.MR), cm(rom.fR), cm(rom.CR)]
    Vc = cm(V) if V is not None else None
    sh = np.ascontiguousarray(np.asarray(shifts_hz, dtype=np.float64))
    lo, hi = np.array([band[0]], np.float64), np.array([band[1]], np.float64)
    kk, ns = np.array([k], np.int32), np.array([sh.size], np.int32)
    st = L.fsi_rom_store()
    st.info = L.fsi_rom_info(nwin=1, kmax=k, nrhs=int(rom.fR.shape[1]), nrcv=int(rom.CR.shape[0]),
                             n=int(V.shape[0]) if V is not None else 0, nshift_total=int(sh.size))
    st.on_device = 1
    st.KR, st.DR, st.MR, st.fR, st.CR = [_ptr(b) for b in bufs]
    st.V = _ptr(Vc) if Vc is not None else None
    st.lo, st.hi = lo.ctypes.data_as(L.c_double_p), hi.ctypes.data_as(L.c_double_p)
    st.k, st.nshift = kk.ctypes.data_as(L.c_int32_p), ns.ctypes.data_as(L.c_int32_p)
    st.shifts_hz = sh.ctypes.data_as(L.c_double_p) if sh.size else None
    L.check(lib.rom_save(path.encode(), C.byref(st), _stream_ptr()), "rom_save")


def rom_file_info(path: str) -> L.fsi_rom_info:
    info = L.fsi_rom_info()
    L.check(L.load().rom_file_info(path.encode(), C.byref(info)), "rom_file_info")
    return info


def rom_load(path: str):
    """Read a one-window reduced model saved by rom_save: (DeviceROM, shifts_hz, V or None, band)."""
    torch = _torch()
    lib = L.load()
    info = rom_file_info(path)
    if info.nwin != 1:
        raise ValueError("rom_load reads one-window files; this one has %d windows" % info.nwin)
    k, nrhs, nrcv, n = info.kmax, info.nrhs, info.nrcv, int(info.n)
    dev = dict(dtype=torch.complex128, device="cuda")
    KR, DR, MR = (torch.empty((k, k), **dev) for _ in range(3))
    fR = torch.empty((nrhs, k), **dev)
    CR = torch.empty((k, nrcv), **dev)
    V = torch.empty((k, n), **dev) if n > 0 else None
    sh = np.zeros(max(info.nshift_total, 1), np.float64)
    lo, hi = np.zeros(1), np.zeros(1)
    kk, ns = np.zeros(1, np.int32), np.zeros(1, np.int32)
    st = L.fsi_rom_store()
    st.info = info
    st.on_device = 1
    st.KR, st.DR, st.MR, st.fR, st.CR = _ptr(KR), _ptr(DR), _ptr(MR), _ptr(fR), _ptr(CR)
    st.V = _ptr(V) if V is not None else None
    st.lo, st.hi = lo.ctypes.data_as(L.c_double_p), hi.ctypes.data_as(L.c_double_p)
    st.k, st.nshift = kk.ctypes.data_as(L.c_int32_p), ns.ctypes.data_as(L.c_int32_p)
    st.shifts_hz = sh.ctypes.data_as(L.c_double_p)
    L.check(lib.rom_load(path.encode(), C.byref(st), _stream_ptr()), "rom_load")
    rom = DeviceROM(KR=KR.t(), DR=DR.t(), MR=MR.t(), fR=fR.t(), CR=CR.t())
    return rom, sh[:int(ns[0])].copy(), (V.t() if V is not None else None), (float(lo[0]), float(hi[0]))


@dataclass
class GreedyResult:
    V: object            # n x k basis (torch, device)
    rom: DeviceROM
    shifts_hz: np.ndarray
    est: np.ndarray      # residual estimate at every candidate (last round)
    history: np.ndarray  # largest estimate per round


def rom_greedy(model: DeviceModel, F, rcv, cand_hz, q: int, kmax: int, max_shifts: int, tol: float,
               init_hz=None, precision="fp32_ir", max_refine=10, refine_tol=1e-10,
               second_order=-1, mlp_params=None, batch_shifts=1) -> GreedyResult:
    """Greedy expansion points with the Gram-block residual estimate (C-ABI rom_greedy)."""
    torch = _torch()
    lib = L.load()
    cand = np.ascontiguousarray(np.asarray(cand_hz, dtype=np.float64))
    init = np.ascontiguousarray(np.asarray([] if init_hz is None else init_hz, dtype=np.float64))
    n = int(model.dims.n)
    nrhs = F.shape[1]
    o = L.fsi_greedy_opts()
    o.q, o.kmax, o.max_shifts, o.tol = int(q), int(kmax), int(max_shifts), float(tol)
    o.build = _rom_opts(precision, max_refine, refine_tol, second_order, batch_shifts)
    o.mlp = _ptr(mlp_params) if mlp_params is not None else None
    need = C.c_size_t()
    L.check(lib.rom_greedy_workspace(C.byref(model.dims), nrhs, C.byref(o), C.byref(need)), "rom_greedy_workspace")
    ws = torch.empty(need.value, dtype=torch.uint8, device="cuda")
    Fc = F.t().contiguous()
    r = rcv.to(torch.int32).contiguous()
    nrcv = int(r.numel())
    Vt = torch.zeros((kmax, n), dtype=torch.complex128, device="cuda")
    KR = torch.empty(kmax * kmax, dtype=torch.complex128, device="cuda")
    DR = torch.empty_like(KR)
    MR = torch.empty_like(KR)
    fR = torch.empty(kmax * nrhs, dtype=torch.complex128, device="cuda")
    CR = torch.empty(kmax * nrcv, dtype=torch.complex128, device="cuda")
    k = C.c_int(0)
    ns = C.c_int(0)
    shifts = np.zeros(max_shifts, np.float64)
    est = np.zeros(cand.size, np.float64)
    hist = np.zeros(max_shifts, np.float64)
    L.check(lib.rom_greedy(C.byref(model.dims), _ptr(model.buf), _ptr(Fc), nrhs, cand.ctypes.data_as(L.c_double_p),
                           int(cand.size), init.ctypes.data_as(L.c_double_p), int(init.size), C.byref(o), _ptr(ws),
                           C.c_size_t(need.value), _ptr(Vt), C.byref(k), _ptr(KR), _ptr(DR), _ptr(MR), _ptr(fR),
                           _ptr(r), nrcv, _ptr(CR), shifts.ctypes.data_as(L.c_double_p), C.byref(ns),
                           est.ctypes.data_as(L.c_double_p), hist.ctypes.data_as(L.c_double_p), _stream_ptr()),
            "rom_greedy")
    kk, nsh = k.value, ns.value
    cm = lambda buf, r_, c_: buf[:r_ * c_].view(c_, r_).t()   # column-major r_ x c_ buffer as a matrix
    rom = DeviceROM(KR=cm(KR, kk, kk), DR=cm(DR, kk, kk), MR=cm(MR, kk, kk), fR=cm(fR, kk, nrhs),
                    CR=cm(CR, nrcv, kk))
    nrounds = nsh - max(int(init.size), 1) + 1
    return GreedyResult(V=Vt[:kk].t(), rom=rom, shifts_hz=shifts[:nsh].copy(), est=est,
                        history=hist[:max(nrounds, 0)].copy())


@dataclass
class WindowedROM:
    lo: np.ndarray        # first candidate of each window (Hz)
    hi: np.ndarray        # last candidate of each window
    k: np.ndarray         # basis columns per window
    nshift: np.ndarray    # expansion points per window
    maxest: np.ndarray    # largest final residual estimate per window
    nreused: np.ndarray   # expansion points reused from enclosing windows (no new factorisation)
    kmax: int
    nrhs: int
    nrcv: int
    bufs: tuple           # device slots (KR, DR, MR, fR, CR)


def rom_windows(model: DeviceModel, F, rcv, cand_hz, q: int, kmax: int, max_shifts: int, tol: float,
                max_windows: int = 16, min_points: int = 4, precision="fp32_ir", max_refine=10,
                refine_tol=1e-10, second_order=-1, reuse: bool = True, batch_shifts=1, init_points=0,
                init_windows=1) -> WindowedROM:
    """Local ROMs over windows of the candidate band (C-ABI rom_windows); with reuse, a window
    split from a larger one starts from that window's expansion points in its band."""
    torch = _torch()
    lib = L.load()
    cand = np.ascontiguousarray(np.asarray(cand_hz, dtype=np.float64))
    nrhs = F.shape[1]
    o = L.fsi_window_opts()
    o.greedy.q, o.greedy.kmax, o.greedy.max_shifts, o.greedy.tol = int(q), int(kmax), int(max_shifts), float(tol)
    o.greedy.build = _rom_opts(precision, max_refine, refine_tol, second_order, batch_shifts)
    o.max_windows, o.min_points, o.reuse = int(max_windows), int(min_points), int(bool(reuse))
    o.init_points, o.init_windows = int(init_points), int(init_windows)
    need = C.c_size_t()
    L.check(lib.rom_windows_workspace(C.byref(model.dims), nrhs, C.byref(o), C.byref(need)), "rom_windows_workspace")
    ws = torch.empty(need.value, dtype=torch.uint8, device="cuda")
    Fc = F.t().contiguous()
    r = rcv.to(torch.int32).contiguous()
    nrcv = int(r.numel())
    W = int(max_windows)
    KR = torch.empty(W * kmax * kmax, dtype=torch.complex128, device="cuda")
    DR = torch.empty_like(KR)
    MR = torch.empty_like(KR)
    fR = torch.empty(W * kmax * nrhs, dtype=torch.complex128, device="cuda")
    CR = torch.empty(W * nrcv * kmax, dtype=torch.complex128, device="cuda")
    nw = C.c_int(0)
    lo, hi, mx = np.zeros(W), np.zeros(W), np.zeros(W)
    kk, ns, nr = np.zeros(W, np.int32), np.zeros(W, np.int32), np.zeros(W, np.int32)
    L.check(lib.rom_windows(C.byref(model.dims), _ptr(model.buf), _ptr(Fc), nrhs, cand.ctypes.data_as(L.c_double_p),
                            int(cand.size), C.byref(o), _ptr(ws), C.c_size_t(need.value), _ptr(r), nrcv, _ptr(KR),
                            _ptr(DR), _ptr(MR), _ptr(fR), _ptr(CR), C.byref(nw), lo.ctypes.data_as(L.c_double_p),
                            hi.ctypes.data_as(L.c_double_p), kk.ctypes.data_as(L.c_int32_p),
                            ns.ctypes.data_as(L.c_int32_p), mx.ctypes.data_as(L.c_double_p),
                            nr.ctypes.data_as(L.c_int32_p), _stream_ptr()),
            "rom_windows")
    n = nw.value
    del ws
    return WindowedROM(lo=lo[:n].copy(), hi=hi[:n].copy(), k=kk[:n].copy(), nshift=ns[:n].copy(),
                       maxest=mx[:n].copy(), nreused=nr[:n].copy(), kmax=int(kmax), nrhs=nrhs, nrcv=nrcv,
                       bufs=(KR, DR, MR, fR, CR))


def rom_windows_sweep(wr: WindowedROM, freqs_hz, batch: int = 256):
    """Receiver pressures and SPL [nf][nrcv][nrhs] from windowed ROMs (torch, device)."""
    torch = _torch()
    lib = L.load()
    f = np.ascontiguousarray(np.asarray(freqs_hz, dtype=np.float64))
    nf = int(f.size)
    bt = min(batch, nf)
    need = C.c_size_t()
    L.check(lib.rom_windows_sweep_workspace(wr.kmax, wr.nrhs, bt, C.byref(need)), "rom_windows_sweep_workspace")
    ws = torch.empty(need.value, dtype=torch.uint8, device="cuda")
    p = torch.empty((nf, wr.nrcv, wr.nrhs), dtype=torch.complex128, device="cuda")
    spl = torch.empty((nf, wr.nrcv, wr.nrhs), dtype=torch.float64, device="cuda")
    lo = np.ascontiguousarray(wr.lo)
    hi = np.ascontiguousarray(wr.hi)
    k = np.ascontiguousarray(wr.k.astype(np.int32))
    KR, DR, MR, fR, CR = wr.bufs
    L.check(lib.rom_windows_sweep(len(k), lo.ctypes.data_as(L.c_double_p), hi.ctypes.data_as(L.c_double_p),
                                  k.ctypes.data_as(L.c_int32_p), wr.kmax, _ptr(KR), _ptr(DR), _ptr(MR), _ptr(fR),
                                  _ptr(CR), wr.nrhs, wr.nrcv, f.ctypes.data_as(L.c_double_p), nf, bt, _ptr(ws),
                                  C.c_size_t(need.value), _ptr(p), _ptr(spl), _stream_ptr()), "rom_windows_sweep")
    return p, spl


@dataclass
class MlpState:
    params: object   # FP32 master parameters (torch, device)
    m: object        # Adam moments
    v: object
    steps: int = 0


def mlp_state(init_params) -> MlpState:
    """Estimator state from flat initial parameters (numpy or torch)."""
    torch = _torch()
    p = torch.as_tensor(np.asarray(init_params, dtype=np.float32), device="cuda").contiguous()
    assert p.numel() == L.MLP_PARAMS
    return MlpState(params=p, m=torch.zeros_like(p), v=torch.zeros_like(p))


def mlp_train(state: MlpState, X, T, order, lr: float = 1e-3, want_grad: bool = False):
    """Adam steps over the batches order (steps x batch) of rows of X (n x 5), T (n);
    returns per-step losses (and the last step's gradient)."""
    torch = _torch()
    lib = L.load()
    Xd = torch.as_tensor(np.asarray(X, dtype=np.float32), device="cuda").contiguous()
    Td = torch.as_tensor(np.asarray(T, dtype=np.float32), device="cuda").contiguous()
    od = torch.as_tensor(np.asarray(order, dtype=np.int32), device="cuda").contiguous()
    steps, batch = int(od.shape[0]), int(od.shape[1])
    losses = torch.empty(steps, dtype=torch.float32, device="cuda")
    grad = torch.empty(L.MLP_PARAMS, dtype=torch.float32, device="cuda") if want_grad else None
    L.check(lib.mlp_train(_ptr(state.params), _ptr(state.m), _ptr(state.v), _ptr(Xd), _ptr(Td), int(Xd.shape[0]),
                          _ptr(od), steps, batch, C.c_float(lr), state.steps, _ptr(losses),
                          _ptr(grad) if grad is not None else None, _stream_ptr()), "mlp_train")
    state.steps += steps
    return (losses, grad) if want_grad else losses


def rom_output_error(p_ref, p):
    """Relative output error per frequency of p against p_ref ([nf][nrcv][nrhs] complex, device)."""
    torch = _torch()
    lib = L.load()
    a = p_ref.contiguous()
    b = p.contiguous()
    nf = int(a.shape[0])
    err = torch.empty(nf, dtype=torch.float64, device=a.device)
    L.check(lib.rom_output_error(_ptr(a), _ptr(b), nf, int(a[0].numel()), _ptr(err), _stream_ptr()),
            "rom_output_error")
    return err


def rom_features(cand_hz, shifts_hz, est, lo: float, hi: float) -> np.ndarray:
    """Estimator features at the candidates (n x 5 float32, host)."""
    lib = L.load()
    c = np.ascontiguousarray(np.asarray(cand_hz, dtype=np.float64))
    sh = np.ascontiguousarray(np.asarray(shifts_hz, dtype=np.float64))
    e = np.ascontiguousarray(np.asarray(est, dtype=np.float64))
    X = np.empty((c.size, 5), np.float32)
    L.check(lib.rom_features(c.ctypes.data_as(L.c_double_p), int(c.size), sh.ctypes.data_as(L.c_double_p),
                             int(sh.size), e.ctypes.data_as(L.c_double_p), float(lo), float(hi),
                             X.ctypes.data_as(C.c_void_p)), "rom_features")
    return X


def mlp_predict(params, X):
    """Network outputs for the rows of X (n x 5)."""
    torch = _torch()
    lib = L.load()
    Xd = torch.as_tensor(np.asarray(X, dtype=np.float32), device="cuda").contiguous()
    y = torch.empty(int(Xd.shape[0]), dtype=torch.float32, device="cuda")
    L.check(lib.mlp_predict(_ptr(params), _ptr(Xd), int(Xd.shape[0]), _ptr(y), _stream_ptr()), "mlp_predict")
    return y


class MultiSweep:
    """Reduced sweeps of several ROMs in one persistent launch (C-ABI rom_multi_sweep).

    Buffers (descriptors, prefix sums, queue counter, outputs) are made once; launch()
    only enqueues device work on the current stream, so it can be captured into a
    CUDA graph and replayed.  Models are queued in order of decreasing k."""

    def __init__(self, roms: Sequence[DeviceROM], freqs: Sequence[Sequence[float]]):
        torch = _torch()
        assert len(roms) == len(freqs) and len(roms) > 0
        cm = lambda X: X.t().contiguous()
        self.order = sorted(range(len(roms)), key=lambda i: -roms[i].k)
        self._keep = []
        self.p = [None] * len(roms)
        self.spl = [None] * len(roms)
        items = (L.fsi_rom_item * len(roms))()
        off = [0]
        for slot, i in enumerate(self.order):
            r = roms[i]
            if r.k > 128 or r.fR.shape[1] > 4:
                raise ValueError("rom_multi_sweep handles k <= 128 and at most 4 load columns")
            f = torch.as_tensor(np.asarray(freqs[i], dtype=np.float64), device="cuda")
            nf, nrcv, nrhs = int(f.numel()), int(r.CR.shape[0]), int(r.fR.shape[1])
            bufs = (cm(r.KR), cm(r.DR), cm(r.MR), cm(r.fR), cm(r.CR), f)
            self.p[i] = torch.empty((nf, nrcv, nrhs), dtype=torch.complex128, device="cuda")
            self.spl[i] = torch.empty((nf, nrcv, nrhs), dtype=torch.float64, device="cuda")
            self._keep.append(bufs)
            it = items[slot]
            it.k, it.nrhs, it.nrcv, it.nf = r.k, nrhs, nrcv, nf
            it.KR, it.DR, it.MR, it.fR, it.CR, it.f_hz = (b.data_ptr() for b in bufs)
            it.p_out, it.spl_out = self.p[i].data_ptr(), self.spl[i].data_ptr()
            off.append(off[-1] + nf)
        raw = bytes(items)
        self.items = torch.tensor(list(raw), dtype=torch.uint8, device="cuda")
        self.offsets = torch.tensor(off, dtype=torch.int32, device="cuda")
        self.total = off[-1]
        self.counter = torch.zeros(1, dtype=torch.int32, device="cuda")
        self.status = torch.zeros(self.total, dtype=torch.int32, device="cuda")
        self.nvar = len(roms)

    def launch(self):
        lib = L.load()
        L.check(lib.rom_multi_sweep(_ptr(self.items), self.nvar, _ptr(self.offsets), self.total, _ptr(self.counter),
                                    _ptr(self.status), _stream_ptr()), "rom_multi_sweep")

    def fixup(self, roms, freqs) -> int:
        """Re-solve with the FP64 reduced sweep the items whose refinement did not converge
        (status 3); returns their number.  Items with a singular pivot stay flagged."""
        st = self.status.cpu().numpy()
        off = self.offsets.cpu().numpy()
        fixed = 0
        for slot, i in enumerate(self.order):
            bad = np.nonzero(st[off[slot]:off[slot + 1]] == 3)[0]
            if bad.size == 0:
                continue
            f = np.asarray(freqs[i], dtype=np.float64)[bad]
            p, spl = rom_sweep(roms[i], f, batch=max(1, min(64, bad.size)))
            idx = _torch().as_tensor(bad, device="cuda")
            self.p[i][idx] = p
            self.spl[i][idx] = spl
            fixed += int(bad.size)
        return fixed


def load_matrix_dofs(spec, loads, n_rhs):
    """Load columns as (DoF index, column, value) triplets for the slab-major numbering."""
    npl = spec.nx * spec.ny
    b = npl + 3 * (2 * (spec.nx - 1) + 2 * (spec.ny - 1))
    return [(ld.slab * b + npl + 3 * ld.ring, ld.column, ld.value) for ld in loads]


def dense_loads(spec, loads, n_rhs, device="cuda"):
    """n x nrhs complex128 load matrix on the device."""
    torch = _torch()
    npl = spec.nx * spec.ny
    b = npl + 3 * (2 * (spec.nx - 1) + 2 * (spec.ny - 1))
    F = torch.zeros((b * spec.nz, n_rhs), dtype=torch.complex128, device=device)
    for g, c, v in load_matrix_dofs(spec, loads, n_rhs):
        F[g, c] += complex(v)
    return F


def receiver_dofs(spec, receivers) -> np.ndarray:
    npl = spec.nx * spec.ny
    b = npl + 3 * (2 * (spec.nx - 1) + 2 * (spec.ny - 1))
    return np.array([k * b + i + spec.nx * j for (i, j, k) in receivers], dtype=np.int32)
