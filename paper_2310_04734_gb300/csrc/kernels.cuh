// Device-side types, complex helpers and kernel launchers (internal).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace fsi {

// Device view of the model buffer written by fsi_assemble.
struct DevModel {
    const int32_t* rowptr;
    const int32_t* col;
    const double2* K;
    const double* M;
    const double2* D;
    const double* kdiag;
    const double* cbase;   // scale factors without their w dependence (negative on fluid rows)
    const double* rbase;
    int64_t n;
    int b, nz, npl;
    double rho;
};

template <typename R>
struct Cplx;
template <>
struct Cplx<float> {
    using T = float2;
};
template <>
struct Cplx<double> {
    using T = double2;
};

template <typename T2>
__host__ __device__ __forceinline__ T2 mk(decltype(T2::x) re, decltype(T2::x) im) {
    T2 r;
    r.x = re;
    r.y = im;
    return r;
}
template <typename T2>
__device__ __forceinline__ T2 cadd(T2 a, T2 b) { return mk<T2>(a.x + b.x, a.y + b.y); }
template <typename T2>
__device__ __forceinline__ T2 csub(T2 a, T2 b) { return mk<T2>(a.x - b.x, a.y - b.y); }
template <typename T2>
__device__ __forceinline__ T2 cmul(T2 a, T2 b) { return mk<T2>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
// acc += a * b
template <typename T2>
__device__ __forceinline__ void cfma(T2& acc, T2 a, T2 b) {
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(-a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y);
    acc.y = fma(a.y, b.x, acc.y);
}
// acc -= a * b
template <typename T2>
__device__ __forceinline__ void cfms(T2& acc, T2 a, T2 b) {
    acc.x = fma(-a.x, b.x, acc.x);
    acc.x = fma(a.y, b.y, acc.x);
    acc.y = fma(-a.x, b.y, acc.y);
    acc.y = fma(-a.y, b.x, acc.y);
}
// 1 / a with scaling against overflow (Smith's method)
template <typename T2>
__device__ __forceinline__ T2 cinv(T2 a) {
    using R = decltype(T2::x);
    if (fabs(a.x) >= fabs(a.y)) {
        R r = a.y / a.x, d = a.x + a.y * r;
        return mk<T2>(R(1) / d, -r / d);
    } else {
        R r = a.x / a.y, d = a.x * r + a.y;
        return mk<T2>(r / d, R(-1) / d);
    }
}

// Scaling of the equilibrated system  (R A C) y = R f,  x = C y :
// the fluid rows are divided by rho w^2 (reciprocity symmetrisation), then a
// symmetric Jacobi scaling by |K_ii|^-1/2 is applied.
__device__ __forceinline__ bool is_fluid(const DevModel& m, int64_t g) { return (g % m.b) < m.npl; }
// (the fluid/shell test reads the sign bit on the integer pipe: FP64 compares share
// GB300's narrow FP64 pipe with the arithmetic)
__device__ __forceinline__ bool neg_bits(double v) { return __double_as_longlong(v) < 0; }
__device__ __forceinline__ double row_scale(const DevModel& m, int64_t g, double w) {
    const double r = m.rbase[g];   // fluid: 1/(w sqrt(rho |K_ii|)), shell: 1/sqrt(|K_ii|)
    return neg_bits(r) ? -r / w : r;
}
// row_scale with 1/w precomputed (a multiply instead of an FP64 divide per row)
__device__ __forceinline__ double row_scale_inv(const DevModel& m, int64_t g, double inv_w) {
    const double r = m.rbase[g];
    return neg_bits(r) ? -r * inv_w : r;
}
__device__ __forceinline__ double col_scale(const DevModel& m, int64_t g, double w) {
    const double c = m.cbase[g];   // fluid: w sqrt(rho / |K_ii|), shell: 1/sqrt(|K_ii|)
    return neg_bits(c) ? -c * w : c;
}
// A(w)_e = K_e + i w D_e - w^2 M_e
__device__ __forceinline__ double2 a_entry(const DevModel& m, int64_t e, double w) {
    const double2 k = m.K[e], d = m.D[e];
    const double mm = m.M[e];
    return make_double2(k.x - w * d.y - w * w * mm, k.y + w * d.x);
}

// ------------------------------------------------------------------ launchers
// All batched over F matrices / frequencies; `s*` are element strides between batch members.

// Dense scaled rows of A(w_f): rows of slab `row_slab` into rows [g_row0, g_row0+b) of G,
// columns [col_slab0*b, col_slab0*b + wcols) of A into columns [0, wcols).
template <typename R>
void launch_form_rows(const DevModel& m, typename Cplx<R>::T* G, int64_t sG, int ld, int F,
                      const double* d_omega, int row_slab, int g_row0, int col_slab0, int wcols,
                      cudaStream_t st);

// Unblocked LU with partial pivoting of the panel rows [j0, m) x cols [j0, j0+nbw); its row
// interchanges are applied to the columns [c0, j0) and [j0+nbw, c1) as well.
template <typename R>
void launch_panel(typename Cplx<R>::T* G, int64_t sG, int ld, int F, int m, int j0, int nbw,
                  int32_t* ipiv, int64_t sP, int32_t* status, int c0, int c1, cudaStream_t st);
// Row interchanges ipiv[j..j+cnt) on columns [a0,a1) and [b0,b1).
template <typename R>
void launch_laswp(typename Cplx<R>::T* G, int64_t sG, int ld, int F, int j, int cnt, const int32_t* ipiv,
                  int64_t sP, int a0, int a1, int b0, int b1, cudaStream_t st);
// Rows [j, j+cnt), columns [c0,c1): B <- L^-1 B with L the unit lower block at (j, j).
template <typename R>
void launch_trsm(typename Cplx<R>::T* G, int64_t sG, int ld, int F, int j, int cnt, int c0, int c1,
                 cudaStream_t st);
// G[r0:r1, c0:c1] -= G[r0:r1, k0:k0+K] * G[k0:k0+K, c0:c1]
template <typename R>
void launch_gemm_update(typename Cplx<R>::T* G, int64_t sG, int ld, int F, int r0, int r1, int c0, int c1,
                        int k0, int K, cudaStream_t st);

// Tensor-core trailing updates: device error flag (set to 1 when a bounded wait gave up) and the
// workspace that holds the split operands of one update.
struct TcCtx {
    int32_t* err = nullptr;
    void* ws = nullptr;
    size_t ws_bytes = 0;
    int planes = 3;   // BF16 planes per operand: 3 (six products, FP32 level) or 1 (plain BF16)
    size_t a_bytes = 0;   // the first a_bytes of ws hold the A operand of one update
    // the U12 columns [bc0, bc0 + bN) of the current slab step, packed block by block after ws + a_bytes
    void* bpack = nullptr;
    int64_t bKp = 0;
    int bN = 0, bc0 = 0;
};
// Workspace bytes for every trailing update of partial_lu(F, m, ncols, npiv) on the tensor cores,
// and the part of it that holds the A operand of one update.
size_t tc_workspace_bytes(int F, int m, int ncols, int npiv, int planes);
size_t tc_a_region_bytes(int F, int m, int ncols, int npiv, int planes);
// Columns [c0, c1) right of the npiv pivots: prepare the packed U12 operand (false: the tensor-core
// path does not apply; use launch_tc_update / the SIMT update).  Then tc_pack_b_rows packs rows
// [k_begin, k_end) of U12 once they are final, and launch_tc_update_lazy runs
// C[r0:r1, c0:c1] -= A[r0:r1, k0:k0+K] U12[k0:k0+K, c0:c1] from the packed rows (2 k0 a multiple
// of 64; false: not launched).
bool tc_begin_lazy(float2* G, int64_t sG, int ld, int F, int npiv, int c0, int c1, TcCtx& tc, cudaStream_t st);
void tc_pack_b_rows(float2* G, int64_t sG, int ld, int F, int k_begin, int k_end, const TcCtx& tc, cudaStream_t st);
bool launch_tc_update_lazy(float2* G, int64_t sG, int ld, int F, int r0, int r1, int k0, int K, const TcCtx& tc,
                           cudaStream_t st);
// Spin limit of the tensor-core kernels' pipeline waits (0: the default, about 6.7e7 polls).
void set_tc_spin_limit(uint32_t spins);
// Trailing update C -= A B of the FP32 band LU on tcgen05 tensor cores (BF16 planes, TMA-fed).
// Returns false (nothing launched) when the operands do not meet TMA's alignment rules or the
// workspace is too small; the caller then runs the SIMT update.
bool launch_tc_update(float2* G, int64_t sG, int ld, int F, int r0, int r1, int c0, int c1, int k0, int K,
                      const TcCtx& tc, cudaStream_t st);

// Batched partial LU driver on device matrices (uses the kernels above).  With tc != NULL
// (FP32 only) the large trailing updates run on the tensor cores.
template <typename R>
int panel_width(int m);
template <typename R>
void partial_lu(typename Cplx<R>::T* G, int64_t sG, int ld, int F, int m, int ncols, int npiv,
                int32_t* ipiv, int64_t sP, int32_t* status, cudaStream_t st, const TcCtx* tc = nullptr);

// After a slab step: save factor rows and multipliers, turn ipiv into a row
// permutation of the stacked rows, and move the Schur tail to the top rows.
template <typename R>
void launch_slab_shift(typename Cplx<R>::T* G, int64_t sG, int F, int b, int m, typename Cplx<R>::T* U,
                       int64_t sU, typename Cplx<R>::T* L, int64_t sL, const int32_t* ipiv, int64_t sP,
                       int32_t* perm, int64_t sPerm, cudaStream_t st);

// Complex FP32 C[r0:r1, c0:c1] -= A[r0:r1, k0:k0+K] B[k0:k0+K, c0:c1] in each of F matrices (SIMT).
void launch_cgemm_f32(float2* G, int64_t sG, int ld, int F, int r0, int r1, int c0, int c1, int k0, int K,
                      cudaStream_t st);

// Slab solves: per slab a triangle launch (one CTA per frequency) and a batched
// matrix-vector launch for the off-diagonal factor blocks.  F frequencies are
// solved: 0..F-1, or flist[0..F) when flist (device) is non-null.
template <typename R>
void launch_slab_solve_fwd(const typename Cplx<R>::T* U, const typename Cplx<R>::T* L, int64_t sU, int64_t sL,
                           const int32_t* perm, int64_t sPerm, typename Cplx<R>::T* y, int64_t sY, int64_t n, int b,
                           int k, int nz, int nrhs, int F, const int32_t* flist, cudaStream_t st);
template <typename R>
void launch_slab_solve_bwd(const typename Cplx<R>::T* U, int64_t sU, typename Cplx<R>::T* y, int64_t sY, int64_t n,
                           int b, int k, int nz, int nrhs, int F, const int32_t* flist, cudaStream_t st);

// U x = B in place for the upper triangle of the first n columns; B = columns [c0, c0+nrhs).
template <typename R>
void launch_backsub(typename Cplx<R>::T* G, int64_t sG, int ld, int F, int n, int c0, int nrhs, cudaStream_t st);

// FP64 residual r = rs o (F - A(w_f) (cs o x)) (scaled) or F - A x (unscaled);
// x may be NULL (x = 0).  Accumulates |r|^2 per (f, column) into norms if non-NULL.
// omega per batch member from d_omega, or the scalar omega0 when d_omega is NULL.
// absn (optional) accumulates |rs o (|A| |cs o x| + |F|)|^2 per (f, column): the size of the
// terms whose FP64 rounding bounds the attainable residual.  sF: stride between the
// frequencies' right-hand sides (0: Fm is shared by all of them).
void launch_residual(const DevModel& m, const double* d_omega, double omega0, int F, const double2* x,
                     int64_t sX, const double2* Fm, int nrhs, double2* r, int64_t sR, double* norms,
                     bool scaled, cudaStream_t st, double* absn = nullptr, int64_t sF = 0);
// y = (T)(r / s) with s = sqrt(norms) per (f, column)
template <typename R>
void launch_to_low(const double2* r, int64_t sR, const double* norms, typename Cplx<R>::T* y, int64_t sY,
                   int64_t n, int nrhs, int F, cudaStream_t st);
// x += s * y for active (f, column)
template <typename R>
void launch_update(double2* x, int64_t sX, const double* norms, const typename Cplx<R>::T* y, int64_t sY,
                   int64_t n, int nrhs, int F, const int32_t* active, cudaStream_t st);
// p[f][i][c] = cs(rcv_i) * x[f][c][rcv_i], spl
void launch_receivers(const DevModel& m, const double* d_omega, int F, const double2* x, int64_t sX,
                      const int32_t* rcv, int nrcv, int nrhs, double2* p, double* spl, cudaStream_t st);

}  // namespace fsi
