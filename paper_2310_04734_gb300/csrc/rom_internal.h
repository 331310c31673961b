// Internal interface between the ROM build / reduced sweep (rom.cu) and the
// greedy expansion-point selection (rom_greedy.cu).
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include "fsi_internal.h"

namespace fsi {

// Krylov blocks of expansion points kept for reuse by later builds (the windows of one
// rom_windows call): block b holds ncol columns at buf + col0 * n spanning the point's own
// moment space (first order: its local Arnoldi basis; second order: the SOAR bases of its
// load columns).  [lo, hi) is the candidate index range of the window that computed it.
struct MomentBlock {
    double shift;
    int64_t col0;
    int ncol;
    int lo, hi;
};
struct MomentStore {
    double2* buf = nullptr;   // n x cap columns
    int64_t cap = 0, used = 0;
    int lo = 0, hi = 0;       // owner range recorded with new blocks
    std::vector<MomentBlock> blocks;
};

// Workspace of rom_build_append (factor of one expansion point + moment buffers).
template <typename R>
size_t rom_build_ws(const fsi_dims& d, int nrhs, int q, int kmax, const fsi_rom_opts& o);

// Rational Arnoldi moments at the given expansion points appended to the k_in
// orthonormal columns already in V (n x kmax, column-major); *k_out = columns after.
// With a store, each point's Krylov block is also recorded there (while it has room).
template <typename R>
fsi_status rom_build_append(const fsi_dims& d, const void* d_model, const double* shifts, int nshift, int q,
                            const double2* F, int nrhs, int kmax, const fsi_rom_opts& o, void* ws, size_t ws_bytes,
                            double2* V, int k_in, int* k_out, cudaStream_t st, MomentStore* store = nullptr);

// CGS2-append ncol columns (n x ncol, column-major, left unchanged) to V[:, :k] (deflated
// columns are dropped, at most kmax in all); scratch of rom_append_ws(n, kmax) bytes.
size_t rom_append_ws(int64_t n, int kmax);
fsi_status rom_append_columns(double2* V, int64_t n, int& k, int kmax, const double2* cols, int ncol, void* ws,
                              size_t ws_bytes, cudaStream_t st);

// Solutions of Fb reduced systems (K_R + i w D_R - w^2 M_R) x_R = f_R, w = 2 pi f_hz[i]:
// x_R[f][j][c] = cs[f*k + j] * G[f*k*(k+nrhs) + j*(k+nrhs) + k + c]  (equilibrated dense LU, FP64).
struct ReducedBatch {
    double2* G = nullptr;
    double* cs = nullptr;
    double* omega = nullptr;   // device, Fb
    int k = 0, nrhs = 0, F = 0;
};
size_t reduced_solve_ws(int k, int nrhs, int batch);
fsi_status reduced_solve_batch(int k, const double2* KR, const double2* DR, const double2* MR, const double2* fR,
                               int nrhs, const double* f_hz, int Fb, void* ws, size_t ws_bytes, ReducedBatch& out,
                               cudaStream_t st);

// p[f][ir][c] = C_R x_R (and SPL when spl is non-null) for the batch's frequencies.
fsi_status reduced_receivers(const ReducedBatch& rb, const double2* CR, int nrcv, double2* p, double* spl,
                             cudaStream_t st);

}  // namespace fsi
