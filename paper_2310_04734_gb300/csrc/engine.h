// Host-side factor / solve engine shared by the full-order sweep and the ROM build.
#pragma once

#include <vector>

#include "fsi_internal.h"
#include "kernels.cuh"

namespace fsi {

DevModel dev_model(const fsi_dims& d, const void* blob);

// ------------------------------------------------------------------ factor / solve engine
// Per-batch buffers of one block-banded factorisation.
template <typename R>
struct Factor {
    using T2 = typename Cplx<R>::T;
    T2* G = nullptr;
    T2* U = nullptr;
    T2* L = nullptr;
    int32_t* ipiv = nullptr;
    int32_t* perm = nullptr;
    int32_t* status = nullptr;
    TcCtx tc;                    // tensor-core updates (FP32 storage only): error flag, operand packs
    bool use_tc = false;
    int64_t sG = 0, sU = 0, sL = 0, sP = 0, sPerm = 0;

    // planes: 0 (no tensor-core updates), 3 (BF16x6, FP32 level) or 1 (plain BF16)
    void carve(Carver& c, const fsi_dims& d, int F, int nrhs, int planes = 0) {
        const int64_t b = d.b, nz = d.nz;
        sG = 2 * b * 3 * b;
        sU = nz * b * 3 * b;
        sL = nz * b * b;
        sP = nz * b;
        sPerm = nz * 2 * b;
        G = c.take<T2>(size_t(F) * sG);
        U = c.take<T2>(size_t(F) * sU);
        L = c.take<T2>(size_t(F) * sL);
        ipiv = c.take<int32_t>(size_t(F) * sP);
        perm = c.take<int32_t>(size_t(F) * sPerm);
        status = c.take<int32_t>(size_t(F));
        tc.err = c.take<int32_t>(1);
        if (planes > 0 && sizeof(R) == 4) {
            tc.planes = planes;
            tc.ws_bytes = tc_workspace_bytes(F, 2 * d.b, 3 * d.b, d.b, planes);
            tc.a_bytes = tc_a_region_bytes(F, 2 * d.b, 3 * d.b, d.b, planes);
            tc.ws = c.take<char>(tc.ws_bytes);
        }
    }
};


// A scaled residual below kResFloor * u64 * |rs o (|A| |cs o x| + |F|)| is at the
// rounding level of its own FP64 evaluation (and of a backward-stable FP64 solve):
// refinement cannot reduce it further, so a pair there counts as converged even
// if its relative residual is above the requested tolerance.
constexpr double kResFloor = 8.0 * 1.1102230246251565e-16;

template <typename R>
fsi_status factor_batch(const DevModel& m, Factor<R>& fc, int F, const double* d_omega, cudaStream_t st);

// Iterative refinement of A(w_f) x = B for every batch member: FP64 scaled
// residual, correction by the stored factors in precision R.  On return xhat
// holds the scaled solution (x = cs o xhat); it_done[f] is the first iteration
// whose relative residual reached tol or the rounding floor (-1: neither), rel[f]
// the last relative residual.  absn: F*nrhs scratch for the floor.  sB: stride between the
// frequencies' right-hand sides in Bdev (0: one right-hand side block for all of them).
template <typename R>
fsi_status ir_solve(const DevModel& m, Factor<R>& fc, int Fb, const double* d_omega, const double2* Bdev, int nrhs,
                    double2* xhat, double2* rhat, typename Cplx<R>::T* y, double* norms, double* fnorms,
                    double* absn, int64_t sV, int max_it, double tol, std::vector<int>& it_done, std::vector<double>& rel, cudaStream_t st,
                    int64_t sB = 0);

// Forward and backward slab solves of y (F frequencies, nrhs columns each, stride sY);
// with flist (device, nF entries) only the listed frequencies are solved.
template <typename R>
fsi_status solve_batch(const DevModel& m, Factor<R>& fc, int F, typename Cplx<R>::T* y, int64_t sY, int nrhs,
                       cudaStream_t st, const int32_t* flist = nullptr, int nF = 0);

// Flexible GMRES on the FP64 scaled system, right preconditioned by the factor in
// precision R, restarted every `restart` iterations, at most max_cycles cycles;
// same outputs as ir_solve (it_done counts preconditioned solves).
size_t gmres_ws_bytes(int64_t n, int P, int restart);
template <typename R>
fsi_status fgmres_solve(const DevModel& m, Factor<R>& fc, int Fb, const double* d_omega, const double2* Bdev,
                        int nrhs, double2* xhat, double2* rhat, typename Cplx<R>::T* y, double* norms, double* fnorms,
                        double* absn, int64_t sV, int restart, int max_cycles, double tol, void* gws, size_t gws_bytes,
                        std::vector<int>& it_done, std::vector<double>& rel, cudaStream_t st);

}  // namespace fsi
