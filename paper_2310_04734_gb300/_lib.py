"""ctypes view of ``libfsi.so`` (the C ABI in include/fsi.h).

Loading fails loudly when the library has not been built: there is no
fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfsi.so")

c_void_p = C.c_void_p
c_int = C.c_int
c_int32_p = C.POINTER(C.c_int32)
c_double_p = C.POINTER(C.c_double)
c_size_t = C.c_size_t


class fsi_c64(C.Structure):
    _fields_ = [("re", C.c_double), ("im", C.c_double)]


class fsi_model_desc(C.Structure):
    _fields_ = [("Lx", C.c_double), ("Ly", C.c_double), ("Lz", C.c_double),
                ("nx", c_int), ("ny", c_int), ("nz", c_int),
                ("c", C.c_double), ("rho", C.c_double),
                ("E", C.c_double), ("nu", C.c_double), ("rho_s", C.c_double), ("t", C.c_double),
                ("eta", c_double_p), ("n_eta", c_int),
                ("has_floor", c_int), ("Z_re", C.c_double), ("Z_im", C.c_double)]


class fsi_dims(C.Structure):
    _fields_ = [("n", C.c_int64), ("b", c_int), ("nz", c_int), ("n_press_slab", c_int),
                ("n_ring", c_int), ("nnz", C.c_int64), ("model_bytes", c_size_t), ("rho", C.c_double)]


class fsi_solve_opts(C.Structure):
    _fields_ = [("precision", c_int), ("batch", c_int), ("max_refine", c_int), ("tol", C.c_double),
                ("host_io", c_int), ("profile", c_int), ("refine", c_int), ("restart", c_int)]


class fsi_sweep_stats(C.Structure):
    _fields_ = [("n_done", c_int), ("max_iters", c_int), ("max_relres", C.c_double),
                ("n_unconverged", c_int), ("launches", C.c_int64), ("kernel_ms", C.c_double * 12),
                ("kernel_flops", C.c_double * 12), ("kernel_launches", C.c_int64 * 12)]


MLP_PARAMS = 4609


class fsi_rom_opts(C.Structure):
    _fields_ = [("precision", c_int), ("max_refine", c_int), ("tol", C.c_double),
                ("second_order", c_int), ("batch_shifts", c_int)]


class fsi_greedy_opts(C.Structure):
    _fields_ = [("q", c_int), ("kmax", c_int), ("max_shifts", c_int), ("tol", C.c_double),
                ("build", fsi_rom_opts), ("mlp", c_void_p)]


class fsi_window_opts(C.Structure):
    _fields_ = [("greedy", fsi_greedy_opts), ("max_windows", c_int), ("min_points", c_int), ("reuse", c_int),
                ("init_points", c_int), ("init_windows", c_int)]


class fsi_rom_item(C.Structure):
    _fields_ = [("k", c_int), ("nrhs", c_int), ("nrcv", c_int), ("nf", c_int), ("KR", c_void_p), ("DR", c_void_p),
                ("MR", c_void_p), ("fR", c_void_p), ("CR", c_void_p), ("f_hz", c_void_p), ("p_out", c_void_p),
                ("spl_out", c_void_p)]


class fsi_rom_info(C.Structure):
    _fields_ = [("nwin", c_int), ("kmax", c_int), ("nrhs", c_int), ("nrcv", c_int), ("n", C.c_int64),
                ("nshift_total", c_int)]


class fsi_rom_store(C.Structure):
    _fields_ = [("info", fsi_rom_info), ("on_device", c_int), ("KR", c_void_p), ("DR", c_void_p), ("MR", c_void_p),
                ("fR", c_void_p), ("CR", c_void_p), ("V", c_void_p), ("lo", c_double_p), ("hi", c_double_p),
                ("k", c_int32_p), ("nshift", c_int32_p), ("shifts_hz", c_double_p)]


# name -> (restype, argtypes)
SIGNATURES = {
    "fsi_model_dims": (c_int, [C.POINTER(fsi_model_desc), C.POINTER(fsi_dims)]),
    "fsi_assemble_host": (c_int, [C.POINTER(fsi_model_desc), c_int32_p, c_int32_p, c_void_p,
                                  c_double_p, c_void_p]),
    "fsi_assemble": (c_int, [C.POINTER(fsi_model_desc), c_void_p, c_size_t, c_void_p]),
    "frf_sweep_workspace": (c_int, [C.POINTER(fsi_dims), C.POINTER(fsi_solve_opts), c_int, c_int,
                                    C.POINTER(c_size_t)]),
    "frf_sweep_full": (c_int, [C.POINTER(fsi_dims), c_void_p, c_double_p, c_int, c_void_p, c_int,
                               c_void_p, c_int, C.POINTER(fsi_solve_opts), c_void_p, c_size_t,
                               c_void_p, c_void_p, c_int32_p, c_double_p,
                               C.POINTER(fsi_sweep_stats), c_void_p]),
    "fsi_residual": (c_int, [C.POINTER(fsi_dims), c_void_p, c_double_p, c_int, c_void_p, c_void_p,
                             c_int, c_void_p, c_void_p]),
    "fsi_lu_workspace": (c_int, [c_int, c_int, c_int, c_int, c_int, C.POINTER(c_size_t)]),
    "fsi_set_wait_limit": (c_int, [C.c_int64]),
    "fsi_batched_lu": (c_int, [c_int, c_int, c_int, c_int, c_int, c_void_p, C.c_int64, C.c_int64,
                               c_void_p, c_void_p, c_size_t, C.POINTER(c_int), c_void_p]),
    "fsi_batched_lu_noalloc": (c_int, [c_int, c_int, c_int, c_int, c_int, c_void_p, C.c_int64, C.c_int64,
                                       c_void_p, C.POINTER(c_int), c_void_p]),
    "rom_workspace": (c_int, [C.POINTER(fsi_dims), c_int, c_int, c_int, C.POINTER(fsi_rom_opts),
                              C.POINTER(c_size_t)]),
    "rom_build": (c_int, [C.POINTER(fsi_dims), c_void_p, c_double_p, c_int, c_int, c_void_p, c_int,
                          c_int, C.POINTER(fsi_rom_opts), c_void_p, c_size_t, c_void_p,
                          C.POINTER(c_int), c_void_p]),
    "rom_project": (c_int, [C.POINTER(fsi_dims), c_void_p, c_void_p, c_int, c_void_p, c_int, c_void_p,
                            c_int, c_void_p, c_size_t, c_void_p, c_void_p, c_void_p, c_void_p,
                            c_void_p, c_void_p]),
    "rom_sweep_workspace": (c_int, [c_int, c_int, c_int, c_int, c_int, C.POINTER(c_size_t)]),
    "rom_sweep": (c_int, [c_int, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_int, c_int,
                          c_double_p, c_int, c_int, c_int, c_void_p, c_size_t, c_void_p, c_void_p, c_int32_p,
                          c_void_p]),
    "rom_residual_check_workspace": (c_int, [C.POINTER(fsi_dims), c_int, c_int, c_int, C.POINTER(c_size_t)]),
    "rom_residual_check": (c_int, [C.POINTER(fsi_dims), c_void_p, c_void_p, c_int, c_void_p, c_void_p, c_void_p,
                                   c_void_p, c_void_p, c_int, c_double_p, c_int, c_int, c_void_p, c_size_t,
                                   c_double_p, c_void_p]),
    "rom_check_resolve_workspace": (c_int, [C.POINTER(fsi_dims), c_int, c_int, c_int, c_int,
                                            C.POINTER(fsi_solve_opts), C.POINTER(c_size_t)]),
    "rom_check_resolve": (c_int, [C.POINTER(fsi_dims), c_void_p, c_void_p, c_int, c_void_p, c_void_p, c_void_p,
                                  c_void_p, c_void_p, c_int, c_void_p, c_int, c_double_p, c_int, c_int, C.c_double,
                                  C.POINTER(fsi_solve_opts), c_void_p, c_size_t, c_void_p, c_void_p, c_double_p,
                                  c_int32_p, C.POINTER(c_int), c_void_p]),
    "rom_save": (c_int, [C.c_char_p, C.POINTER(fsi_rom_store), c_void_p]),
    "rom_file_info": (c_int, [C.c_char_p, C.POINTER(fsi_rom_info)]),
    "rom_load": (c_int, [C.c_char_p, C.POINTER(fsi_rom_store), c_void_p]),
    "rom_greedy_workspace": (c_int, [C.POINTER(fsi_dims), c_int, C.POINTER(fsi_greedy_opts),
                                     C.POINTER(c_size_t)]),
    "rom_greedy": (c_int, [C.POINTER(fsi_dims), c_void_p, c_void_p, c_int, c_double_p, c_int, c_double_p,
                           c_int, C.POINTER(fsi_greedy_opts), c_void_p, c_size_t, c_void_p, C.POINTER(c_int),
                           c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_int, c_void_p, c_double_p,
                           C.POINTER(c_int), c_double_p, c_double_p, c_void_p]),
    "rom_windows_workspace": (c_int, [C.POINTER(fsi_dims), c_int, C.POINTER(fsi_window_opts),
                                      C.POINTER(c_size_t)]),
    "rom_windows": (c_int, [C.POINTER(fsi_dims), c_void_p, c_void_p, c_int, c_double_p, c_int,
                            C.POINTER(fsi_window_opts), c_void_p, c_size_t, c_void_p, c_int, c_void_p, c_void_p,
                            c_void_p, c_void_p, c_void_p, C.POINTER(c_int), c_double_p, c_double_p, c_int32_p,
                            c_int32_p, c_double_p, c_int32_p, c_void_p]),
    "rom_windows_sweep_workspace": (c_int, [c_int, c_int, c_int, C.POINTER(c_size_t)]),
    "rom_windows_sweep": (c_int, [c_int, c_double_p, c_double_p, c_int32_p, c_int, c_void_p, c_void_p, c_void_p,
                                  c_void_p, c_void_p, c_int, c_int, c_double_p, c_int, c_int, c_void_p, c_size_t,
                                  c_void_p, c_void_p, c_void_p]),
    "rom_output_error": (c_int, [c_void_p, c_void_p, c_int, c_int, c_void_p, c_void_p]),
    "rom_features": (c_int, [c_double_p, c_int, c_double_p, c_int, c_double_p, C.c_double, C.c_double, c_void_p]),
    "rom_multi_sweep": (c_int, [c_void_p, c_int, c_void_p, c_int, c_void_p, c_void_p, c_void_p]),
    "mlp_train": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_int, c_void_p, c_int, c_int,
                          C.c_float, c_int, c_void_p, c_void_p, c_void_p]),
    "mlp_predict": (c_int, [c_void_p, c_void_p, c_int, c_void_p, c_void_p]),
    "fsi_probe_peak": (c_int, [c_int, C.c_double, c_void_p, c_double_p, c_double_p, c_void_p]),
    "fsi_status_str": (C.c_char_p, [c_int]),
    "fsi_last_error": (C.c_char_p, []),
}

_LIB = None


def load() -> C.CDLL:
    """Load libfsi.so (raises if it is missing: build it with __graft_entry__.build())."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing; build the CUDA library first "
                               "(python -c 'import __graft_entry__ as g; g.build()')")
        lib = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _LIB = lib
    return _LIB


class FsiError(RuntimeError):
    def __init__(self, status: int, where: str):
        lib = load()
        msg = lib.fsi_last_error().decode(errors="replace")
        super().__init__(f"{where}: {lib.fsi_status_str(status).decode()} ({status}): {msg}")
        self.status = status


def check(status: int, where: str):
    if status != 0:
        raise FsiError(status, where)
