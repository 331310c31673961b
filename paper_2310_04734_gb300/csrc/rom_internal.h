// Internal interface between the ROM build / reduced sweep (rom.cu) and the
// greedy expansion-point selection (rom_greedy.cu).
#pragma once

#include <cuda_runtime.h>

#include "fsi_internal.h"

namespace fsi {

// Workspace of rom_build_append (factor of one expansion point + moment buffers).
template <typename R>
size_t rom_build_ws(const fsi_dims& d, int nrhs, int q, int kmax);

// Rational Arnoldi moments at the given expansion points appended to the k_in
// orthonormal columns already in V (n x kmax, column-major); *k_out = columns after.
template <typename R>
fsi_status rom_build_append(const fsi_dims& d, const void* d_model, const double* shifts, int nshift, int q,
                            const double2* F, int nrhs, int kmax, const fsi_rom_opts& o, void* ws, size_t ws_bytes,
                            double2* V, int k_in, int* k_out, cudaStream_t st);

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
