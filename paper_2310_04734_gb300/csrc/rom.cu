// Rational Arnoldi model order reduction (paper Sec. 3.3, Eq. 9-11).
//
// rom_build  : per expansion point w_j, factor Kt_j = A(w_j) once (the
//              block-banded engine of the full-order sweep, batch of one) and
//              generate q moments per load column from it -- first order
//              (Eq. 10) v <- Kt_j^-1 M v, or second order (Eq. 9) by the SOAR
//              recurrence with A = -Kt_j^-1 Dt_j, B = -Kt_j^-1 M, Dt_j = 2 i w_j M
//              + D.  Every solve is refined against the FP64 residual.  Each
//              new vector is orthonormalised against the basis by classical
//              Gram-Schmidt applied twice (CGS2) and dropped when its norm
//              after both passes is below 1e-10 of its norm before.
// rom_project: K_R = V^H K V, D_R, M_R (sparse-times-dense, then a split-K
//              V^H X product), f_R = V^H F, C_R = rows of V at the receivers.
// rom_sweep  : batched reduced systems K_R + i w D_R - w^2 M_R, equilibrated
//              (row, then column max scaling), dense LU with partial pivoting
//              in FP64 (the same batched kernels as the full-order factor),
//              back substitution, receivers and SPL.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <sstream>
#include <string>
#include <vector>

#include "csr_rows.cuh"
#include "engine.h"
#include "fsi_internal.h"
#include "kernels.cuh"
#include "rom_internal.h"

namespace fsi {

#define ROM_CUDA(call)                                                                                 \
    do {                                                                                               \
        cudaError_t e_ = (call);                                                                       \
        if (e_ != cudaSuccess) {                                                                       \
            std::ostringstream o_;                                                                     \
            o_ << #call << ": " << cudaGetErrorString(e_) << " (" << __FILE__ << ":" << __LINE__ << ")"; \
            set_error(o_.str());                                                                       \
            return FSI_ECUDA;                                                                          \
        }                                                                                              \
    } while (0)
#define ROM_LAUNCH() ROM_CUDA(cudaGetLastError())
#define ROM_REQUIRE(cond, msg) \
    do {                       \
        if (!(cond)) {         \
            set_error(msg);    \
            return FSI_EINVAL; \
        }                      \
    } while (0)

namespace {

constexpr int kChunks = 64;       // row chunks of the V^H w reductions
constexpr int kSplit = 16;        // split-K factor of the V^H X projection
constexpr int kSpC = 4;           // columns per row group in the projection products
constexpr double kDeflate = 1e-10;

inline unsigned cdiv(int64_t a, int64_t b) { return unsigned((a + b - 1) / b); }

// y[c] = sum_e (cK K_e + cD D_e + cM M_e) x[c][col_e]  (unscaled, column-major n x nrhs),
// column c = blockIdx.y; row groups of kRowLanes lanes (lane 0 of a group writes)
__global__ void __launch_bounds__(kRowThreads) spmv_kernel(DevModel m, double2 cK, double2 cD, double2 cM,
                                                           const double2* x, double2* y, int nrhs, bool accumulate) {
    const int c = blockIdx.y;
    if (c >= nrhs) return;
    const int g = threadIdx.x & (kRowLanes - 1);
    const double2* xc = x + c * m.n;
    for (int64_t base = int64_t(blockIdx.x) * kRowsPerCta; base < m.n; base += int64_t(gridDim.x) * kRowsPerCta) {
        const int64_t i = base + threadIdx.x / kRowLanes;
        const bool valid = i < m.n;
        double2 acc = make_double2(0.0, 0.0);
        if (valid) {
            const int e1 = __ldg(m.rowptr + i + 1);
            for (int e = __ldg(m.rowptr + i) + g; e < e1; e += kRowLanes) {
                const double2 k = __ldg(m.K + e), d = __ldg(m.D + e);
                const double mm = __ldg(m.M + e);
                double2 a = cmul(cK, k);
                a = cadd(a, cmul(cD, d));
                a.x = fma(cM.x, mm, a.x);
                a.y = fma(cM.y, mm, a.y);
                cfma(acc, a, xc[__ldg(m.col + e)]);
            }
        }
        acc = group_sum(acc);
        if (valid && g == 0) {
            if (accumulate) acc = cadd(acc, y[c * m.n + i]);
            y[c * m.n + i] = acc;
        }
    }
}

// Back-projection of a batch of reduced solutions: x[f][c][i] = sum_j V[i][j] x_R[f][j][c] with
// x_R[f][j][c] = cs[f*k + j] G[f*k*(k+nrhs) + j*(k+nrhs) + k + c] (the equilibrated reduced
// solve's layout); frequency f = blockIdx.y, one thread per row, columns c < nrhs <= NR
template <int NR>
__global__ void backproject_kernel(const double2* V, int64_t n, int k, const double2* G, const double* cs, int nrhs,
                                   double2* x) {
    const int f = blockIdx.y;
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int ld = k + nrhs;
    const double2* Gf = G + int64_t(f) * k * ld;
    const double* csf = cs + int64_t(f) * k;
    double2 acc[NR];
#pragma unroll
    for (int c = 0; c < NR; ++c) acc[c] = make_double2(0.0, 0.0);
    for (int j = 0; j < k; ++j) {
        const double2 v = V[int64_t(j) * n + i];
        const double s = __ldg(csf + j);
#pragma unroll
        for (int c = 0; c < NR; ++c)
            if (c < nrhs) {
                const double2 g = __ldg(Gf + int64_t(j) * ld + k + c);
                cfma(acc[c], v, make_double2(s * g.x, s * g.y));
            }
    }
#pragma unroll
    for (int c = 0; c < NR; ++c)
        if (c < nrhs) x[(int64_t(f) * nrhs + c) * n + i] = acc[c];
}

unsigned spmv_grid_x(int64_t n, int ncols) {
    static const int per_sm = resident_ctas(spmv_kernel);
    return row_grid_x(n, ncols, per_sm);
}

// partial[chunk][j][c] = sum_{i in chunk} conj(V[i][j]) W[i][c], c < nrhs <= NR.  NR is a
// template bound: the column loop is unrolled to NR, and columns at or above nrhs are
// predicated off but still issue on the FP64 pipe, so the single-column CGS2 of the basis
// build runs the NR = 1 instance.
template <int NR>
__global__ void gram_partial_kernel(const double2* V, int64_t n, int k, const double2* W, int nrhs,
                                    double2* partial) {
    const int j = blockIdx.x, chunk = blockIdx.y;
    const int64_t len = (n + kChunks - 1) / kChunks;
    const int64_t i0 = chunk * len, i1 = min(n, i0 + len);
    double2 acc[NR];
#pragma unroll
    for (int c = 0; c < NR; ++c) acc[c] = make_double2(0.0, 0.0);
    const double2* vj = V + int64_t(j) * n;
    for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
        const double2 v = vj[i];
        const double2 vc = make_double2(v.x, -v.y);
#pragma unroll
        for (int c = 0; c < NR; ++c)
            if (c < nrhs) cfma(acc[c], vc, W[c * n + i]);
    }
    __shared__ double2 red[NR][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int c = 0; c < NR; ++c) {
        if (c >= nrhs) break;
        for (int off = 16; off > 0; off >>= 1) {
            acc[c].x += __shfl_down_sync(0xffffffffu, acc[c].x, off);
            acc[c].y += __shfl_down_sync(0xffffffffu, acc[c].y, off);
        }
        if (lane == 0) red[c][warp] = acc[c];
    }
    __syncthreads();
    if (threadIdx.x < nrhs) {
        double2 s = make_double2(0.0, 0.0);
        for (int w = 0; w < int(blockDim.x >> 5); ++w) s = cadd(s, red[threadIdx.x][w]);
        partial[(int64_t(chunk) * k + j) * nrhs + threadIdx.x] = s;
    }
}

// H[j][c] = sum_chunks partial
__global__ void gram_reduce_kernel(const double2* partial, int k, int nrhs, double2* H) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= k * nrhs) return;
    double2 s = make_double2(0.0, 0.0);
    for (int ch = 0; ch < kChunks; ++ch) s = cadd(s, partial[int64_t(ch) * k * nrhs + q]);
    H[q] = s;
}

// W[i][c] -= sum_j V[i][j] H[j][c], c < nrhs <= NR (NR as for gram_partial_kernel)
template <int NR>
__global__ void cgs_update_kernel(const double2* V, int64_t n, int k, const double2* H, int nrhs, double2* W) {
    extern __shared__ double2 Hs[];
    for (int q = threadIdx.x; q < k * nrhs; q += blockDim.x) Hs[q] = H[q];
    __syncthreads();
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double2 acc[NR];
#pragma unroll
    for (int c = 0; c < NR; ++c) acc[c] = make_double2(0.0, 0.0);
    for (int j = 0; j < k; ++j) {
        const double2 v = V[int64_t(j) * n + i];
#pragma unroll
        for (int c = 0; c < NR; ++c)
            if (c < nrhs) cfma(acc[c], v, Hs[j * nrhs + c]);
    }
#pragma unroll
    for (int c = 0; c < NR; ++c)
        if (c < nrhs) W[c * n + i] = csub(W[c * n + i], acc[c]);
}

void launch_gram_partial(const double2* V, int64_t n, int k, const double2* W, int nrhs, double2* partial,
                         cudaStream_t st) {
    if (nrhs == 1)
        gram_partial_kernel<1><<<dim3(k, kChunks), 256, 0, st>>>(V, n, k, W, nrhs, partial);
    else
        gram_partial_kernel<8><<<dim3(k, kChunks), 256, 0, st>>>(V, n, k, W, nrhs, partial);
}

void launch_cgs_update(const double2* V, int64_t n, int k, const double2* H, int nrhs, double2* W, cudaStream_t st) {
    const size_t smem = size_t(k) * nrhs * sizeof(double2);
    if (nrhs == 1)
        cgs_update_kernel<1><<<cdiv(n, 256), 256, smem, st>>>(V, n, k, H, nrhs, W);
    else
        cgs_update_kernel<8><<<cdiv(n, 256), 256, smem, st>>>(V, n, k, H, nrhs, W);
}

__global__ void sqnorm_kernel(const double2* w, int64_t n, double* out) {
    double s = 0.0;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
        const double2 v = w[i];
        s += v.x * v.x + v.y * v.y;
    }
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
    if ((threadIdx.x & 31) == 0) atomicAdd(out, s);
}

__global__ void axpby_kernel(double2 a, const double2* x, double2 b, const double2* y, double2* out, int64_t n) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double2 r = cmul(a, x[i]);
    if (y) r = cadd(r, cmul(b, y[i]));
    out[i] = r;
}

// x = cs o xhat, scaled by `sign`
__global__ void unscale_kernel(DevModel m, double w, const double2* xhat, double2* x, int nrhs, double sign) {
    const int64_t q = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (q >= m.n * nrhs) return;
    const int64_t i = q % m.n;
    const double s = sign * col_scale(m, i, w);
    x[q] = make_double2(s * xhat[q].x, s * xhat[q].y);
}

// X[j] = A_W V[j] for the projection (A_0 = K, A_1 = D, A_2 = M; columns j = kSpC * blockIdx.y
// + c, c < kSpC, of the n x k product): each entry is loaded once per group of kSpC columns;
// after the reduce-scatter each lane writes its kept columns
template <int W>
__global__ void __launch_bounds__(kRowThreads) spmm_kernel(DevModel m, const double2* V, int k, double2* X) {
    constexpr int KS = kept_slots<kSpC>();
    const int j0 = blockIdx.y * kSpC;
    const int g = threadIdx.x & (kRowLanes - 1);
    const int s0 = slot_base<kSpC>(g);
    const bool writer = slot_writer<kSpC>(g);
    const bool full = j0 + kSpC <= k;   // uniform over the CTA
    for (int64_t base = int64_t(blockIdx.x) * kRowsPerCta; base < m.n; base += int64_t(gridDim.x) * kRowsPerCta) {
        const int64_t i = base + threadIdx.x / kRowLanes;
        const bool valid = i < m.n;
        double2 acc[kSpC];
#pragma unroll
        for (int c = 0; c < kSpC; ++c) acc[c] = make_double2(0.0, 0.0);
        if (valid) {
            const int e1 = __ldg(m.rowptr + i + 1);
            for (int e = __ldg(m.rowptr + i) + g; e < e1; e += kRowLanes) {
                const int64_t col = __ldg(m.col + e);
                const double2 a = W == 0 ? __ldg(m.K + e) : (W == 1 ? __ldg(m.D + e) : make_double2(__ldg(m.M + e), 0.0));
#pragma unroll
                for (int c = 0; c < kSpC; ++c) {
                    // the last column group of a ragged k reads column k - 1 in place of the missing ones
                    const int jc = full ? j0 + c : min(j0 + c, k - 1);
                    const double2 v = V[int64_t(jc) * m.n + col];
                    if (W == 2) {
                        acc[c].x = fma(a.x, v.x, acc[c].x);
                        acc[c].y = fma(a.x, v.y, acc[c].y);
                    } else {
                        cfma(acc[c], a, v);
                    }
                }
            }
        }
        group_reduce_scatter<kSpC>(acc, g);
        if (valid && writer) {
#pragma unroll
            for (int q = 0; q < KS; ++q)
                if (j0 + s0 + q < k) X[int64_t(j0 + s0 + q) * m.n + i] = acc[q];
        }
    }
}

template <int W>
void spmm_launch(const DevModel& m, const double2* V, int k, double2* X, cudaStream_t st) {
    static const int per_sm = resident_ctas(spmm_kernel<W>);
    const int ng = int(cdiv(k, kSpC));
    spmm_kernel<W><<<dim3(row_grid_x(m.n, ng, per_sm), ng), kRowThreads, 0, st>>>(m, V, k, X);
}

// Split-K tile of C = V^H X: partial[s][a][b] over rows of chunk s (32 x 32 tiles, 256 threads).
__global__ void __launch_bounds__(256) vhx_partial_kernel(const double2* V, const double2* X, int64_t n, int k,
                                                          double2* partial) {
    __shared__ double2 Vs[32][33];
    __shared__ double2 Xs[32][33];
    const int ta = blockIdx.x, tb = blockIdx.y, s = blockIdx.z;
    const int64_t len = (n + kSplit - 1) / kSplit;
    const int64_t i0 = s * len, i1 = min(n, i0 + len);
    const int tid = threadIdx.x;
    const int ra = tid >> 3;            // 0..31 output row within tile
    const int cb = (tid & 7) * 4;       // 4 output columns
    double2 acc[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[q] = make_double2(0.0, 0.0);
    for (int64_t base = i0; base < i1; base += 32) {
        for (int idx = tid; idx < 32 * 32; idx += 256) {
            const int col = idx >> 5, ii = idx & 31;
            const int64_t gi = base + ii;
            const int ja = ta * 32 + col, jb = tb * 32 + col;
            Vs[ii][col] = (gi < i1 && ja < k) ? V[int64_t(ja) * n + gi] : make_double2(0.0, 0.0);
            Xs[ii][col] = (gi < i1 && jb < k) ? X[int64_t(jb) * n + gi] : make_double2(0.0, 0.0);
        }
        __syncthreads();
#pragma unroll 8
        for (int ii = 0; ii < 32; ++ii) {
            const double2 v = Vs[ii][ra];
            const double2 vc = make_double2(v.x, -v.y);
#pragma unroll
            for (int q = 0; q < 4; ++q) cfma(acc[q], vc, Xs[ii][cb + q]);
        }
        __syncthreads();
    }
    const int a = ta * 32 + ra;
    if (a >= k) return;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int b = tb * 32 + cb + q;
        if (b < k) partial[(int64_t(s) * k + b) * k + a] = acc[q];   // column-major k x k per split
    }
}

__global__ void split_reduce_kernel(const double2* partial, int64_t kk, double2* C) {
    const int64_t q = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (q >= kk) return;
    double2 s = make_double2(0.0, 0.0);
    for (int p = 0; p < kSplit; ++p) s = cadd(s, partial[p * kk + q]);
    C[q] = s;
}

__global__ void gather_rows_kernel(const double2* V, int64_t n, int k, const int32_t* rcv, int nrcv, double2* CR) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= k * nrcv) return;
    const int j = q / nrcv, ir = q - j * nrcv;
    CR[q] = V[int64_t(j) * n + rcv[ir]];   // column-major nrcv x k
}

// ---- reduced sweep
// G[f] (row-major k x (k+nrhs)) = [A_R(w_f) | f_R] with A_R = K_R + i w D_R - w^2 M_R (column-major inputs)
__global__ void form_reduced_kernel(const double2* KR, const double2* DR, const double2* MR, const double2* fR,
                                    int k, int nrhs, const double* omega, double2* G) {
    const int f = blockIdx.y;
    const int ld = k + nrhs;
    const int64_t q = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (q >= int64_t(k) * ld) return;
    const int i = int(q / ld), j = int(q - int64_t(i) * ld);
    const double w = omega[f];
    double2 v;
    if (j < k) {
        const int64_t e = int64_t(j) * k + i;
        const double2 a = KR[e], d = DR[e], mm = MR[e];
        v = make_double2(a.x - w * d.y - w * w * mm.x, a.y + w * d.x - w * w * mm.y);
    } else {
        v = fR[int64_t(j - k) * k + i];
    }
    G[int64_t(f) * k * ld + q] = v;
}

// row scaling r_i = 1/max_j |a_ij| applied to the whole augmented row (warp per row)
__global__ void row_equil_kernel(double2* G, int k, int nrhs) {
    const int f = blockIdx.y;
    const int ld = k + nrhs;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int i = blockIdx.x * (blockDim.x >> 5) + warp;
    if (i >= k) return;
    double2* row = G + int64_t(f) * k * ld + int64_t(i) * ld;
    double mx = 0.0;
    for (int j = lane; j < k; j += 32) mx = fmax(mx, hypot(row[j].x, row[j].y));
    for (int off = 16; off > 0; off >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, off));
    const double r = mx > 0.0 ? 1.0 / mx : 1.0;
    for (int j = lane; j < ld; j += 32) row[j] = make_double2(row[j].x * r, row[j].y * r);
}

// column scaling c_j = 1/max_i |a_ij| on the first k columns; c saved for the unscaling
__global__ void col_equil_kernel(double2* G, int k, int nrhs, double* cs) {
    const int f = blockIdx.y;
    const int ld = k + nrhs;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= k) return;
    double2* A = G + int64_t(f) * k * ld;
    double mx = 0.0;
    for (int i = 0; i < k; ++i) mx = fmax(mx, hypot(A[int64_t(i) * ld + j].x, A[int64_t(i) * ld + j].y));
    const double c = mx > 0.0 ? 1.0 / mx : 1.0;
    for (int i = 0; i < k; ++i) {
        double2& a = A[int64_t(i) * ld + j];
        a = make_double2(a.x * c, a.y * c);
    }
    cs[int64_t(f) * k + j] = c;
}

// p[f][ir][c] = sum_j C_R[ir][j] cs_j y_j[c]
__global__ void reduced_receivers_kernel(const double2* G, int k, int nrhs, const double* cs, const double2* CR,
                                         int nrcv, double2* p, double* spl) {
    const int f = blockIdx.y;
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nrcv * nrhs) return;
    const int ir = q / nrhs, c = q - ir * nrhs;
    const int ld = k + nrhs;
    const double2* A = G + int64_t(f) * k * ld;
    double2 acc = make_double2(0.0, 0.0);
    for (int j = 0; j < k; ++j) {
        const double2 y = A[int64_t(j) * ld + k + c];
        const double s = cs[int64_t(f) * k + j];
        cfma(acc, CR[int64_t(j) * nrcv + ir], make_double2(s * y.x, s * y.y));
    }
    const int64_t o = (int64_t(f) * nrcv + ir) * nrhs + c;
    p[o] = acc;
    if (spl) spl[o] = 20.0 * log10(sqrt(acc.x * acc.x + acc.y * acc.y) / (sqrt(2.0) * 2e-5));
}

// --------------------------------------------------------------- host helpers
struct CgsBufs {
    double2* partial;
    double2* H;
    double* scal;   // 2 doubles
};

fsi_status sqnorm(const double2* w, int64_t n, double* d_out, double& h_out, cudaStream_t st) {
    ROM_CUDA(cudaMemsetAsync(d_out, 0, sizeof(double), st));
    sqnorm_kernel<<<256, 256, 0, st>>>(w, n, d_out);
    ROM_LAUNCH();
    ROM_CUDA(cudaMemcpyAsync(&h_out, d_out, sizeof(double), cudaMemcpyDeviceToHost, st));
    ROM_CUDA(cudaStreamSynchronize(st));
    return FSI_OK;
}

// H = V[:, :k]^H W (nrhs columns), W -= V H
fsi_status cgs_pass(const double2* V, int64_t n, int k, double2* W, int nrhs, CgsBufs& b, cudaStream_t st) {
    if (k == 0) return FSI_OK;
    launch_gram_partial(V, n, k, W, nrhs, b.partial, st);
    gram_reduce_kernel<<<cdiv(int64_t(k) * nrhs, 256), 256, 0, st>>>(b.partial, k, nrhs, b.H);
    launch_cgs_update(V, n, k, b.H, nrhs, W, st);
    ROM_LAUNCH();
    return FSI_OK;
}

// CGS2-append one column w (device, length n) to V[:, :k].  accepted = whether it was kept.
fsi_status cgs2_append(double2* V, int64_t n, int& k, int kmax, double2* w, CgsBufs& b, bool& accepted,
                       cudaStream_t st) {
    accepted = false;
    if (k >= kmax) return FSI_OK;
    double pre = 0.0, post = 0.0;
    fsi_status s = sqnorm(w, n, b.scal, pre, st);
    if (s != FSI_OK) return s;
    if (!(pre > 0.0)) return FSI_OK;
    for (int pass = 0; pass < 2; ++pass) {
        s = cgs_pass(V, n, k, w, 1, b, st);
        if (s != FSI_OK) return s;
    }
    s = sqnorm(w, n, b.scal, post, st);
    if (s != FSI_OK) return s;
    if (!(std::sqrt(post) > kDeflate * std::sqrt(pre))) return FSI_OK;
    const double inv = 1.0 / std::sqrt(post);
    axpby_kernel<<<cdiv(n, 256), 256, 0, st>>>(make_double2(inv, 0.0), w, make_double2(0.0, 0.0), nullptr,
                                              V + int64_t(k) * n, n);
    ROM_LAUNCH();
    ++k;
    accepted = true;
    return FSI_OK;
}

// expansion points factored and solved together, and BF16 planes of the tensor-core updates
int rom_points(const fsi_rom_opts& o) { return std::max(1, std::min(o.batch_shifts, 64)); }
int rom_planes(const fsi_rom_opts& o) { return o.precision == FSI_BF16X6_IR ? 3 : 0; }

template <typename R>
struct RomWS {
    using T2 = typename Cplx<R>::T;
    Factor<R> fc;
    double* omega;                       // P
    double2 *xhat, *rhat, *X, *B, *W;    // P x sV each (W: n)
    T2* y;                               // P x sV
    double *norms, *fnorms, *absn;       // P x nrhs
    CgsBufs cg;
    double2 *Qs, *Ps;
    double2* Ql;   // local Krylov blocks of P expansion points (first order), P x n x q*nrhs
    int64_t sV;
    int P;

    void carve(Carver& c, const fsi_dims& d, int nrhs, int q, int kmax, int points, int planes) {
        P = points;
        fc.carve(c, d, P, nrhs, planes);
        fc.use_tc = planes > 0;
        sV = int64_t(nrhs) * d.n;
        omega = c.take<double>(P);
        xhat = c.take<double2>(P * sV);
        rhat = c.take<double2>(P * sV);
        X = c.take<double2>(P * sV);
        B = c.take<double2>(P * sV);
        W = c.take<double2>(d.n);
        y = c.take<T2>(P * sV);
        norms = c.take<double>(size_t(P) * nrhs);
        fnorms = c.take<double>(size_t(P) * nrhs);
        absn = c.take<double>(size_t(P) * nrhs);
        const int kk = std::max(kmax, q) + 1;
        cg.partial = c.take<double2>(size_t(kChunks) * kk * std::max(nrhs, 1));
        cg.H = c.take<double2>(size_t(kk) * std::max(nrhs, 1));
        cg.scal = c.take<double>(2);
        Qs = c.take<double2>(size_t(d.n) * q);
        Ps = c.take<double2>(size_t(d.n) * q);
        Ql = c.take<double2>(size_t(P) * d.n * q * nrhs);
    }
};

template <typename R>
size_t rom_ws_bytes(const fsi_dims& d, int nrhs, int q, int kmax, const fsi_rom_opts& o) {
    Carver c(nullptr, 0);
    RomWS<R> w;
    w.carve(c, d, nrhs, q, kmax, rom_points(o), rom_planes(o));
    return align_up(c.used);
}

// x_f = sign * (cs(w_f) o xhat_f) for the F points of a batch
__global__ void unscale_batch_kernel(DevModel m, const double* omega, const double2* xhat, double2* x, int nrhs,
                                     int64_t sV, double sign) {
    const int f = blockIdx.y;
    const int64_t q = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (q >= m.n * nrhs) return;
    const int64_t i = q % m.n;
    const double s = sign * col_scale(m, i, omega[f]);
    const double2 v = xhat[f * sV + q];
    x[f * sV + q] = make_double2(s * v.x, s * v.y);
}

// X = x(w_j) for right-hand sides B (n x nr): refined solve, unscaled, times `sign`.
template <typename R>
fsi_status shifted_solve(const DevModel& m, RomWS<R>& w, double om, const double2* B, int nr, int max_it,
                         double tol, double sign, double2* X, cudaStream_t st) {
    std::vector<int> done;
    std::vector<double> rel;
    fsi_status s = ir_solve<R>(m, w.fc, 1, w.omega, B, nr, w.xhat, w.rhat, w.y, w.norms, w.fnorms, w.absn,
                               int64_t(nr) * m.n, max_it, tol, done, rel, st);
    if (s != FSI_OK) return s;
    unscale_kernel<<<cdiv(m.n * nr, 256), 256, 0, st>>>(m, om, w.xhat, X, nr, sign);
    ROM_LAUNCH();
    return FSI_OK;
}

template <typename R>
fsi_status run_rom_build(const fsi_dims& d, const void* d_model, const double* shifts, int nshift, int q,
                         const double2* F, int nrhs, int kmax, const fsi_rom_opts& o, void* ws, size_t ws_bytes,
                         double2* V, int k_in, int* k_out, cudaStream_t st, MomentStore* store) {
    Carver c(ws, ws_bytes);
    RomWS<R> w;
    w.carve(c, d, nrhs, q, kmax, rom_points(o), rom_planes(o));
    if (!c.fits()) {
        set_error("rom workspace too small");
        return FSI_ENOMEM;
    }
    const DevModel m = dev_model(d, d_model);
    const int64_t n = d.n;
    const int max_it = std::max(1, o.max_refine);
    const double tol = o.tol > 0 ? o.tol : 1e-10;
    // second order (Eq. 9) when the model has a damping matrix, unless forced
    bool second = false;
    if (o.second_order < 0) {
        // D has nonzeros only with a floor impedance; probe |D|^2 through a norm of D * ones
        std::vector<double2> ones_h(size_t(n), make_double2(1.0, 0.0));
        ROM_CUDA(cudaMemcpyAsync(w.B, ones_h.data(), sizeof(double2) * n, cudaMemcpyHostToDevice, st));
        spmv_kernel<<<dim3(spmv_grid_x(n, 1), 1), kRowThreads, 0, st>>>(m, make_double2(0, 0), make_double2(1, 0),
                                                                          make_double2(0, 0), w.B, w.W, 1, false);
        ROM_LAUNCH();
        double dn = 0.0;
        fsi_status s = sqnorm(w.W, n, w.cg.scal, dn, st);
        if (s != FSI_OK) return s;
        second = dn > 0.0;
    } else {
        second = o.second_order != 0;
    }
    int k = k_in;   // columns already in V (orthonormal)
    const int P = second ? 1 : w.P;   // SOAR runs one point at a time
    std::vector<int32_t> hstat(P);
    for (int g0 = 0; g0 < nshift && k < kmax;) {
        const int Pg = std::min(P, nshift - g0);
        std::vector<double> omv(Pg);
        for (int p = 0; p < Pg; ++p) omv[p] = 2.0 * M_PI * shifts[g0 + p];
        const double om = omv[0];
        const int sidx = g0;
        ROM_CUDA(cudaMemcpyAsync(w.omega, omv.data(), sizeof(double) * Pg, cudaMemcpyHostToDevice, st));
        fsi_status s = factor_batch<R>(m, w.fc, Pg, w.omega, st);
        if (s != FSI_OK) return s;
        ROM_CUDA(cudaMemcpyAsync(hstat.data(), w.fc.status, sizeof(int32_t) * Pg, cudaMemcpyDeviceToHost, st));
        ROM_CUDA(cudaStreamSynchronize(st));
        for (int p = 0; p < Pg; ++p)
            if (hstat[p]) {
                set_error("singular shifted matrix at an expansion point");
                return FSI_ESINGULAR;
            }
        g0 += Pg;
        if (!second) {
            // Eq. 10 at Pg points at once: per point a local Arnoldi on Kt^-1 M started from
            // Kt^-1 F (the point's own Krylov space, orthonormalised within the point), the
            // solves of all points batched; afterwards the accepted local vectors of each point,
            // in point order, are CGS2-appended to V
            const int klmax = q * nrhs;
            std::vector<double2*> Ql(Pg);
            std::vector<char> keep(Pg, 0);
            std::vector<int64_t> col0(Pg, 0);
            int64_t next = store ? store->used : 0;
            for (int p = 0; p < Pg; ++p) {
                keep[p] = store && next + klmax <= store->cap;
                col0[p] = keep[p] ? next : 0;
                if (keep[p]) next += klmax;
                Ql[p] = keep[p] ? store->buf + col0[p] * n : w.Ql + int64_t(p) * n * klmax;
            }
            std::vector<int> kl(Pg, 0), nr(Pg, nrhs);
            for (int p = 0; p < Pg; ++p)
                ROM_CUDA(cudaMemcpyAsync(w.B + p * w.sV, F, sizeof(double2) * n * nrhs, cudaMemcpyDeviceToDevice,
                                         st));
            std::vector<int> done;
            std::vector<double> rel;
            for (int mom = 0; mom < q; ++mom) {
                bool any = false;
                for (int p = 0; p < Pg; ++p) any = any || nr[p] > 0;
                if (!any) break;
                s = ir_solve<R>(m, w.fc, Pg, w.omega, w.B, nrhs, w.xhat, w.rhat, w.y, w.norms, w.fnorms, w.absn,
                                w.sV, max_it, tol, done, rel, st, w.sV);
                if (s != FSI_OK) return s;
                unscale_batch_kernel<<<dim3(cdiv(n * nrhs, 256), Pg), 256, 0, st>>>(m, w.omega, w.xhat, w.X, nrhs,
                                                                                   w.sV, 1.0);
                ROM_LAUNCH();
                for (int p = 0; p < Pg; ++p) {
                    const int kl0 = kl[p];
                    for (int cc = 0; cc < nr[p]; ++cc) {
                        bool acc = false;
                        s = cgs2_append(Ql[p], n, kl[p], klmax, w.X + p * w.sV + int64_t(cc) * n, w.cg, acc, st);
                        if (s != FSI_OK) return s;
                    }
                    nr[p] = kl[p] - kl0;
                    double2* Bp = w.B + p * w.sV;
                    if (mom + 1 < q && nr[p] > 0) {
                        spmv_kernel<<<dim3(spmv_grid_x(n, nr[p]), nr[p]), kRowThreads, 0, st>>>(
                            m, make_double2(0, 0), make_double2(0, 0), make_double2(1, 0), Ql[p] + int64_t(kl0) * n,
                            Bp, nr[p], false);
                        ROM_LAUNCH();
                    }
                    if (nr[p] < nrhs)   // columns without a new direction solve zero right-hand sides
                        ROM_CUDA(cudaMemsetAsync(Bp + int64_t(nr[p]) * n, 0, sizeof(double2) * n * (nrhs - nr[p]),
                                                 st));
                }
            }
            for (int p = 0; p < Pg && k < kmax; ++p) {
                for (int j = 0; j < kl[p] && k < kmax; ++j) {
                    ROM_CUDA(cudaMemcpyAsync(w.W, Ql[p] + int64_t(j) * n, sizeof(double2) * n,
                                             cudaMemcpyDeviceToDevice, st));
                    bool acc = false;
                    s = cgs2_append(V, n, k, kmax, w.W, w.cg, acc, st);
                    if (s != FSI_OK) return s;
                }
                // a block cut short by the column budget is not the point's whole Krylov space: not kept
                if (keep[p] && kl[p] > 0 && k < kmax) {
                    store->blocks.push_back(MomentBlock{shifts[sidx + p], col0[p], kl[p], store->lo, store->hi});
                    store->used = col0[p] + kl[p];
                }
            }
            continue;
        }
        // room in the store for this point's block (else the local block stays in the workspace)
        const int64_t blk_cols = int64_t(q) * nrhs;
        const bool keep = store && store->used + blk_cols <= store->cap;
        const int64_t col0 = keep ? store->used : 0;
        int nkept = 0;
        {
            // Eq. 9 by SOAR per load column: q_0 = u/|u|, u = -Kt^-1 f; r = A q_j + B p_j
            const double2 dt = make_double2(0.0, 2.0 * om);   // Dt = D + 2 i w_j M
            for (int cc = 0; cc < nrhs && k < kmax; ++cc) {
                s = shifted_solve<R>(m, w, om, F + int64_t(cc) * n, 1, max_it, tol, -1.0, w.W, st);
                if (s != FSI_OK) return s;
                double nu2 = 0.0;
                s = sqnorm(w.W, n, w.cg.scal, nu2, st);
                if (s != FSI_OK) return s;
                if (!(nu2 > 0.0)) continue;
                const double nu = std::sqrt(nu2);
                axpby_kernel<<<cdiv(n, 256), 256, 0, st>>>(make_double2(1.0 / nu, 0), w.W, make_double2(0, 0),
                                                          nullptr, w.Qs, n);
                ROM_CUDA(cudaMemsetAsync(w.Ps, 0, sizeof(double2) * n, st));
                int nq = 1, ndefl = 0;
                for (int j = 0; j + 1 < q; ++j) {
                    // B = Dt q_j + M p_j ; r = -Kt^-1 B
                    spmv_kernel<<<dim3(spmv_grid_x(n, 1), 1), kRowThreads, 0, st>>>(
                        m, make_double2(0, 0), make_double2(1, 0), dt, w.Qs + int64_t(j) * n, w.B, 1, false);
                    spmv_kernel<<<dim3(spmv_grid_x(n, 1), 1), kRowThreads, 0, st>>>(
                        m, make_double2(0, 0), make_double2(0, 0), make_double2(1, 0), w.Ps + int64_t(j) * n, w.B, 1,
                        true);
                    ROM_LAUNCH();
                    s = shifted_solve<R>(m, w, om, w.B, 1, max_it, tol, -1.0, w.W, st);
                    if (s != FSI_OK) return s;
                    // t = Q^H r ; r -= Q t ; s = q_j - P t
                    double2* sv = w.X;
                    ROM_CUDA(cudaMemcpyAsync(sv, w.Qs + int64_t(j) * n, sizeof(double2) * n, cudaMemcpyDeviceToDevice,
                                             st));
                    launch_gram_partial(w.Qs, n, nq, w.W, 1, w.cg.partial, st);
                    gram_reduce_kernel<<<cdiv(nq, 256), 256, 0, st>>>(w.cg.partial, nq, 1, w.cg.H);
                    launch_cgs_update(w.Qs, n, nq, w.cg.H, 1, w.W, st);
                    launch_cgs_update(w.Ps, n, nq, w.cg.H, 1, sv, st);
                    ROM_LAUNCH();
                    double t2 = 0.0;
                    s = sqnorm(w.W, n, w.cg.scal, t2, st);
                    if (s != FSI_OK) return s;
                    const double t = std::sqrt(t2);
                    if (t > kDeflate * nu) {
                        axpby_kernel<<<cdiv(n, 256), 256, 0, st>>>(make_double2(1.0 / t, 0), w.W,
                                                                  make_double2(0, 0), nullptr,
                                                                  w.Qs + int64_t(j + 1) * n, n);
                        axpby_kernel<<<cdiv(n, 256), 256, 0, st>>>(make_double2(1.0 / t, 0), sv, make_double2(0, 0),
                                                                  nullptr, w.Ps + int64_t(j + 1) * n, n);
                        ROM_LAUNCH();
                    } else {
                        // deflation (Bai and Su): r is in the span already; continue with q = 0 and
                        // p = s, which can still reach new directions, unless s vanishes
                        // (breakdown).  A second deflation in one sequence stops it.
                        double s2 = 0.0;
                        s = sqnorm(sv, n, w.cg.scal, s2, st);
                        if (s != FSI_OK) return s;
                        if (ndefl > 0 || !(std::sqrt(s2) > kDeflate)) break;
                        ++ndefl;
                        ROM_CUDA(cudaMemsetAsync(w.Qs + int64_t(j + 1) * n, 0, sizeof(double2) * n, st));
                        ROM_CUDA(cudaMemcpyAsync(w.Ps + int64_t(j + 1) * n, sv, sizeof(double2) * n,
                                                 cudaMemcpyDeviceToDevice, st));
                    }
                    ++nq;
                }
                if (keep) {
                    ROM_CUDA(cudaMemcpyAsync(store->buf + (col0 + nkept) * n, w.Qs, sizeof(double2) * n * nq,
                                             cudaMemcpyDeviceToDevice, st));
                    nkept += nq;
                }
                for (int j = 0; j < nq && k < kmax; ++j) {
                    ROM_CUDA(cudaMemcpyAsync(w.W, w.Qs + int64_t(j) * n, sizeof(double2) * n, cudaMemcpyDeviceToDevice,
                                             st));
                    bool acc = false;
                    s = cgs2_append(V, n, k, kmax, w.W, w.cg, acc, st);
                    if (s != FSI_OK) return s;
                }
            }
        }
        // a block cut short by the column budget is not the point's whole Krylov space: not kept
        if (keep && nkept > 0 && k < kmax) {
            store->blocks.push_back(MomentBlock{shifts[sidx], col0, nkept, store->lo, store->hi});
            store->used = col0 + nkept;
        }
    }
    ROM_CUDA(cudaStreamSynchronize(st));
    *k_out = k;
    return FSI_OK;
}

}  // namespace

template <typename R>
size_t rom_build_ws(const fsi_dims& d, int nrhs, int q, int kmax, const fsi_rom_opts& o) {
    return rom_ws_bytes<R>(d, nrhs, q, kmax, o);
}

template <typename R>
fsi_status rom_build_append(const fsi_dims& d, const void* d_model, const double* shifts, int nshift, int q,
                            const double2* F, int nrhs, int kmax, const fsi_rom_opts& o, void* ws, size_t ws_bytes,
                            double2* V, int k_in, int* k_out, cudaStream_t st, MomentStore* store) {
    return run_rom_build<R>(d, d_model, shifts, nshift, q, F, nrhs, kmax, o, ws, ws_bytes, V, k_in, k_out, st, store);
}

size_t rom_append_ws(int64_t n, int kmax) {
    Carver c(nullptr, 0);
    c.take<double2>(size_t(kChunks) * (kmax + 1));
    c.take<double2>(size_t(kmax) + 1);
    c.take<double>(2);
    c.take<double2>(size_t(n));
    return align_up(c.used);
}

fsi_status rom_append_columns(double2* V, int64_t n, int& k, int kmax, const double2* cols, int ncol, void* ws,
                              size_t ws_bytes, cudaStream_t st) {
    Carver c(ws, ws_bytes);
    CgsBufs b;
    b.partial = c.take<double2>(size_t(kChunks) * (kmax + 1));
    b.H = c.take<double2>(size_t(kmax) + 1);
    b.scal = c.take<double>(2);
    double2* tmp = c.take<double2>(size_t(n));
    if (!c.fits()) {
        set_error("column append workspace too small");
        return FSI_ENOMEM;
    }
    for (int j = 0; j < ncol && k < kmax; ++j) {
        ROM_CUDA(cudaMemcpyAsync(tmp, cols + int64_t(j) * n, sizeof(double2) * n, cudaMemcpyDeviceToDevice, st));
        bool acc = false;
        fsi_status s = cgs2_append(V, n, k, kmax, tmp, b, acc, st);
        if (s != FSI_OK) return s;
    }
    return FSI_OK;
}

template size_t rom_build_ws<float>(const fsi_dims&, int, int, int, const fsi_rom_opts&);
template size_t rom_build_ws<double>(const fsi_dims&, int, int, int, const fsi_rom_opts&);
template fsi_status rom_build_append<float>(const fsi_dims&, const void*, const double*, int, int, const double2*, int,
                                            int, const fsi_rom_opts&, void*, size_t, double2*, int, int*,
                                            cudaStream_t, MomentStore*);
template fsi_status rom_build_append<double>(const fsi_dims&, const void*, const double*, int, int, const double2*,
                                             int, int, const fsi_rom_opts&, void*, size_t, double2*, int, int*,
                                             cudaStream_t, MomentStore*);

fsi_status reduced_receivers(const ReducedBatch& rb, const double2* CR, int nrcv, double2* p, double* spl,
                             cudaStream_t st) {
    reduced_receivers_kernel<<<dim3(cdiv(int64_t(nrcv) * rb.nrhs, 128), rb.F), 128, 0, st>>>(rb.G, rb.k, rb.nrhs, rb.cs,
                                                                                         CR, nrcv, p, spl);
    ROM_LAUNCH();
    return FSI_OK;
}

size_t reduced_solve_ws(int k, int nrhs, int batch) {
    Carver c(nullptr, 0);
    c.take<double2>(size_t(batch) * k * (k + nrhs));
    c.take<int32_t>(size_t(batch) * k);
    c.take<int32_t>(batch);
    c.take<double>(size_t(batch) * k);
    c.take<double>(batch);
    return align_up(c.used);
}

fsi_status reduced_solve_batch(int k, const double2* KR, const double2* DR, const double2* MR, const double2* fR,
                               int nrhs, const double* f_hz, int Fb, void* ws, size_t ws_bytes, ReducedBatch& out,
                               cudaStream_t st) {
    Carver c(ws, ws_bytes);
    out.G = c.take<double2>(size_t(Fb) * k * (k + nrhs));
    int32_t* ipiv = c.take<int32_t>(size_t(Fb) * k);
    int32_t* status = c.take<int32_t>(Fb);
    out.cs = c.take<double>(size_t(Fb) * k);
    out.omega = c.take<double>(Fb);
    if (!c.fits()) {
        set_error("reduced solve workspace too small");
        return FSI_ENOMEM;
    }
    out.k = k;
    out.nrhs = nrhs;
    out.F = Fb;
    const int ld = k + nrhs;
    std::vector<double> om(Fb);
    std::vector<int32_t> hs(Fb);
    for (int i = 0; i < Fb; ++i) om[i] = 2.0 * M_PI * f_hz[i];
    ROM_CUDA(cudaMemcpyAsync(out.omega, om.data(), sizeof(double) * Fb, cudaMemcpyHostToDevice, st));
    ROM_CUDA(cudaMemsetAsync(status, 0, sizeof(int32_t) * Fb, st));
    form_reduced_kernel<<<dim3(cdiv(int64_t(k) * ld, 256), Fb), 256, 0, st>>>(KR, DR, MR, fR, k, nrhs, out.omega,
                                                                             out.G);
    row_equil_kernel<<<dim3(cdiv(k, 8), Fb), 256, 0, st>>>(out.G, k, nrhs);
    col_equil_kernel<<<dim3(cdiv(k, 128), Fb), 128, 0, st>>>(out.G, k, nrhs, out.cs);
    ROM_LAUNCH();
    partial_lu<double>(out.G, int64_t(k) * ld, ld, Fb, k, ld, k, ipiv, k, status, st);
    launch_backsub<double>(out.G, int64_t(k) * ld, ld, Fb, k, k, nrhs, st);
    ROM_LAUNCH();
    ROM_CUDA(cudaMemcpyAsync(hs.data(), status, sizeof(int32_t) * Fb, cudaMemcpyDeviceToHost, st));
    ROM_CUDA(cudaStreamSynchronize(st));
    for (int i = 0; i < Fb; ++i)
        if (hs[i]) {
            set_error("singular reduced system");
            return FSI_ESINGULAR;
        }
    return FSI_OK;
}

}  // namespace fsi

using namespace fsi;

extern "C" {

fsi_status rom_workspace(const fsi_dims* dims, int nrhs, int q, int kmax, const fsi_rom_opts* opts, size_t* bytes) {
    ROM_REQUIRE(dims && opts && bytes && nrhs > 0 && nrhs <= 8 && q > 0 && kmax > 0, "bad rom workspace arguments");
    ROM_REQUIRE(opts->precision == FSI_FP64 || opts->precision == FSI_FP32_IR || opts->precision == FSI_BF16X6_IR,
                "unknown precision");
    *bytes = opts->precision == FSI_FP64 ? rom_ws_bytes<double>(*dims, nrhs, q, kmax, *opts)
                                         : rom_ws_bytes<float>(*dims, nrhs, q, kmax, *opts);
    return FSI_OK;
}

fsi_status rom_build(const fsi_dims* dims, const void* d_model, const double* shifts_hz, int nshift, int q,
                     const fsi_c64* F, int nrhs, int kmax, const fsi_rom_opts* opts, void* ws, size_t ws_bytes,
                     fsi_c64* V, int* k_out, void* stream) {
    ROM_REQUIRE(dims && d_model && shifts_hz && F && opts && ws && V && k_out, "NULL argument");
    ROM_REQUIRE(nshift > 0 && q > 0 && nrhs > 0 && nrhs <= 8 && kmax > 0 && kmax <= dims->n, "bad rom sizes");
    ROM_REQUIRE(opts->precision == FSI_FP64 || opts->precision == FSI_FP32_IR || opts->precision == FSI_BF16X6_IR,
                "unknown precision");
    for (int i = 0; i < nshift; ++i) ROM_REQUIRE(shifts_hz[i] > 0.0, "expansion points must be > 0 Hz");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const double2* Fd = reinterpret_cast<const double2*>(F);
    double2* Vd = reinterpret_cast<double2*>(V);
    if (opts->precision == FSI_FP64)
        return run_rom_build<double>(*dims, d_model, shifts_hz, nshift, q, Fd, nrhs, kmax, *opts, ws, ws_bytes, Vd, 0,
                                     k_out, st, nullptr);
    return run_rom_build<float>(*dims, d_model, shifts_hz, nshift, q, Fd, nrhs, kmax, *opts, ws, ws_bytes, Vd, 0,
                                k_out, st, nullptr);
}

fsi_status rom_project(const fsi_dims* dims, const void* d_model, const fsi_c64* V, int k, const fsi_c64* F, int nrhs,
                       const int32_t* rcv, int nrcv, void* ws, size_t ws_bytes, fsi_c64* KR, fsi_c64* DR, fsi_c64* MR,
                       fsi_c64* fR, fsi_c64* CR, void* stream) {
    ROM_REQUIRE(dims && d_model && V && F && rcv && ws && KR && DR && MR && fR && CR, "NULL argument");
    ROM_REQUIRE(k > 0 && nrhs > 0 && nrhs <= 8 && nrcv > 0, "bad projection sizes");
    const int64_t n = dims->n;
    Carver c(ws, ws_bytes);
    double2* X = c.take<double2>(size_t(n) * k);
    double2* part = c.take<double2>(size_t(kSplit) * k * k);
    double2* gpart = c.take<double2>(size_t(kChunks) * k * nrhs);
    if (!c.fits()) {
        set_error("rom_project workspace too small: need " + std::to_string(align_up(c.used)) + " bytes");
        return FSI_ENOMEM;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const DevModel m = dev_model(*dims, d_model);
    const double2* Vd = reinterpret_cast<const double2*>(V);
    double2* outs[3] = {reinterpret_cast<double2*>(KR), reinterpret_cast<double2*>(DR), reinterpret_cast<double2*>(MR)};
    for (int which = 0; which < 3; ++which) {
        if (which == 0) spmm_launch<0>(m, Vd, k, X, st);
        else if (which == 1) spmm_launch<1>(m, Vd, k, X, st);
        else spmm_launch<2>(m, Vd, k, X, st);
        vhx_partial_kernel<<<dim3(cdiv(k, 32), cdiv(k, 32), kSplit), 256, 0, st>>>(Vd, X, n, k, part);
        split_reduce_kernel<<<cdiv(int64_t(k) * k, 256), 256, 0, st>>>(part, int64_t(k) * k, outs[which]);
        ROM_LAUNCH();
    }
    // f_R = V^H F (k x nrhs, column-major): H[j][c] layout is row-major k x nrhs -> transpose on copy-out
    double2* H = X;   // reuse
    launch_gram_partial(Vd, n, k, reinterpret_cast<const double2*>(F), nrhs, gpart, st);
    gram_reduce_kernel<<<cdiv(int64_t(k) * nrhs, 256), 256, 0, st>>>(gpart, k, nrhs, H);
    ROM_LAUNCH();
    // explicit transpose (k x nrhs row-major -> column-major)
    for (int cc = 0; cc < nrhs; ++cc)
        ROM_CUDA(cudaMemcpy2DAsync(reinterpret_cast<double2*>(fR) + int64_t(cc) * k, sizeof(double2), H + cc,
                                   sizeof(double2) * nrhs, sizeof(double2), k, cudaMemcpyDeviceToDevice, st));
    gather_rows_kernel<<<cdiv(int64_t(k) * nrcv, 256), 256, 0, st>>>(Vd, n, k, rcv, nrcv,
                                                                       reinterpret_cast<double2*>(CR));
    ROM_LAUNCH();
    ROM_CUDA(cudaStreamSynchronize(st));
    return FSI_OK;
}

// FP32_IR reduced sweep: chunk buffers of the persistent multi-model kernel (one model) and the
// FP64 fallback for frequencies whose refinement stalls.
struct Fp32SweepBufs {
    fsi_rom_item* item;
    int32_t* offs;
    int* counter;
    int32_t* status;
    double* fdev;
    void* fb_ws;
    size_t fb_bytes;
    void carve(Carver& c, int k, int nrhs, int batch) {
        item = c.take<fsi_rom_item>(1);
        offs = c.take<int32_t>(2);
        counter = c.take<int>(1);
        status = c.take<int32_t>(batch);
        fdev = c.take<double>(batch);
        fb_bytes = reduced_solve_ws(k, nrhs, 1);
        fb_ws = c.take<char>(fb_bytes);
    }
};

fsi_status rom_sweep_workspace(int k, int nrhs, int nrcv, int batch, int precision, size_t* bytes) {
    ROM_REQUIRE(k > 0 && nrhs > 0 && nrcv > 0 && batch > 0 && bytes, "bad rom sweep workspace arguments");
    ROM_REQUIRE(precision == FSI_FP64 || precision == FSI_FP32_IR, "unknown precision");
    if (precision == FSI_FP64) {
        *bytes = reduced_solve_ws(k, nrhs, batch);
    } else {
        Carver c(nullptr, 0);
        Fp32SweepBufs b;
        b.carve(c, k, nrhs, batch);
        *bytes = align_up(c.used);
    }
    return FSI_OK;
}

fsi_status rom_sweep(int k, const fsi_c64* KR, const fsi_c64* DR, const fsi_c64* MR, const fsi_c64* fR,
                     const fsi_c64* CR, int nrhs, int nrcv, const double* f_hz, int nf, int batch, int precision,
                     void* ws, size_t ws_bytes, fsi_c64* p_out, double* spl_out, int32_t* fp64_out, void* stream) {
    ROM_REQUIRE(KR && DR && MR && fR && CR && f_hz && ws && p_out, "NULL argument");
    ROM_REQUIRE(k > 0 && k <= 8192 && nrhs > 0 && nrcv > 0 && nf > 0 && batch > 0, "bad rom sweep sizes");
    ROM_REQUIRE(precision == FSI_FP64 || precision == FSI_FP32_IR, "unknown precision");
    ROM_REQUIRE(precision == FSI_FP64 || (k <= 128 && nrhs <= 4),
                "FSI_FP32_IR reduced sweep needs k <= 128 and nrhs <= 4 (use FSI_FP64)");
    const int bt = std::min(batch, nf);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const double2 *K2 = reinterpret_cast<const double2*>(KR), *D2 = reinterpret_cast<const double2*>(DR),
                  *M2 = reinterpret_cast<const double2*>(MR), *f2 = reinterpret_cast<const double2*>(fR),
                  *C2 = reinterpret_cast<const double2*>(CR);
    if (fp64_out) std::fill(fp64_out, fp64_out + nf, 0);
    if (precision == FSI_FP64) {
        for (int f0 = 0; f0 < nf; f0 += bt) {
            const int Fb = std::min(bt, nf - f0);
            ReducedBatch rb;
            fsi_status s = reduced_solve_batch(k, K2, D2, M2, f2, nrhs, f_hz + f0, Fb, ws, ws_bytes, rb, st);
            if (s != FSI_OK) return s;
            s = reduced_receivers(rb, C2, nrcv, reinterpret_cast<double2*>(p_out) + int64_t(f0) * nrcv * nrhs,
                                  spl_out ? spl_out + int64_t(f0) * nrcv * nrhs : nullptr, st);
            if (s != FSI_OK) return s;
        }
        ROM_CUDA(cudaStreamSynchronize(st));
        return FSI_OK;
    }
    Carver c(ws, ws_bytes);
    Fp32SweepBufs b;
    b.carve(c, k, nrhs, bt);
    if (!c.fits()) {
        set_error("rom_sweep workspace too small");
        return FSI_ENOMEM;
    }
    std::vector<int32_t> hs(bt);
    for (int f0 = 0; f0 < nf; f0 += bt) {
        const int Fb = std::min(bt, nf - f0);
        fsi_rom_item it{};
        it.k = k;
        it.nrhs = nrhs;
        it.nrcv = nrcv;
        it.nf = Fb;
        it.KR = KR;
        it.DR = DR;
        it.MR = MR;
        it.fR = fR;
        it.CR = CR;
        it.f_hz = b.fdev;
        it.p_out = p_out + int64_t(f0) * nrcv * nrhs;
        it.spl_out = spl_out ? spl_out + int64_t(f0) * nrcv * nrhs : nullptr;
        const int32_t offs[2] = {0, Fb};
        ROM_CUDA(cudaMemcpyAsync(b.fdev, f_hz + f0, sizeof(double) * Fb, cudaMemcpyHostToDevice, st));
        ROM_CUDA(cudaMemcpyAsync(b.item, &it, sizeof(it), cudaMemcpyHostToDevice, st));
        ROM_CUDA(cudaMemcpyAsync(b.offs, offs, sizeof(offs), cudaMemcpyHostToDevice, st));
        fsi_status s = rom_multi_sweep(b.item, 1, b.offs, Fb, b.counter, b.status, stream);
        if (s != FSI_OK) return s;
        ROM_CUDA(cudaMemcpyAsync(hs.data(), b.status, sizeof(int32_t) * Fb, cudaMemcpyDeviceToHost, st));
        ROM_CUDA(cudaStreamSynchronize(st));   // the host item above stays alive until here
        for (int i = 0; i < Fb; ++i) {
            if (hs[i] == 0) continue;
            // refinement stalled (or a zero FP32 pivot): this frequency again by the FP64 LU
            ReducedBatch rb;
            s = reduced_solve_batch(k, K2, D2, M2, f2, nrhs, f_hz + f0 + i, 1, b.fb_ws, b.fb_bytes, rb, st);
            if (s != FSI_OK) return s;
            s = reduced_receivers(rb, C2, nrcv, reinterpret_cast<double2*>(p_out) + int64_t(f0 + i) * nrcv * nrhs,
                                  spl_out ? spl_out + int64_t(f0 + i) * nrcv * nrhs : nullptr, st);
            if (s != FSI_OK) return s;
            if (fp64_out) fp64_out[f0 + i] = 1;
        }
    }
    ROM_CUDA(cudaStreamSynchronize(st));
    return FSI_OK;
}

fsi_status rom_residual_check_workspace(const fsi_dims* dims, int k, int nrhs, int batch, size_t* bytes) {
    ROM_REQUIRE(dims && bytes && k > 0 && nrhs > 0 && nrhs <= 8 && batch > 0, "bad residual check workspace arguments");
    const size_t vec = size_t(batch) * nrhs * dims->n * sizeof(double2);
    *bytes = reduced_solve_ws(k, nrhs, batch) + 2 * vec + size_t(batch + 1) * nrhs * sizeof(double) + 6 * 256;
    return FSI_OK;
}

fsi_status rom_residual_check(const fsi_dims* dims, const void* d_model, const fsi_c64* V, int k, const fsi_c64* KR,
                              const fsi_c64* DR, const fsi_c64* MR, const fsi_c64* fR, const fsi_c64* F, int nrhs,
                              const double* f_hz, int nf, int batch, void* ws, size_t ws_bytes, double* relres,
                              void* stream) {
    ROM_REQUIRE(dims && d_model && V && KR && DR && MR && fR && F && f_hz && ws && relres, "NULL argument");
    ROM_REQUIRE(k > 0 && k <= dims->n && nrhs > 0 && nrhs <= 8 && nf > 0 && batch > 0, "bad residual check sizes");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const DevModel m = dev_model(*dims, d_model);
    const int64_t n = dims->n;
    const int bt = std::min(batch, nf);
    const size_t red = (reduced_solve_ws(k, nrhs, bt) + 255) & ~size_t(255);
    Carver c(static_cast<char*>(ws) + red, ws_bytes > red ? ws_bytes - red : 0);
    double2* x = c.take<double2>(size_t(bt) * nrhs * n);
    double2* r = c.take<double2>(size_t(bt) * nrhs * n);
    double* norms = c.take<double>(size_t(bt) * nrhs);
    double* fn = c.take<double>(nrhs);
    ROM_REQUIRE(c.fits() && ws_bytes >= red, "residual check workspace too small");
    const double2* Fd = reinterpret_cast<const double2*>(F);
    // |f_c|^2: the residual kernel with no iterate
    ROM_CUDA(cudaMemsetAsync(fn, 0, sizeof(double) * nrhs, st));
    launch_residual(m, nullptr, 1.0, 1, nullptr, 0, Fd, nrhs, r, 0, fn, false, st);
    std::vector<double> hfn(nrhs), hn(size_t(bt) * nrhs);
    ROM_CUDA(cudaMemcpyAsync(hfn.data(), fn, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, st));
    for (int f0 = 0; f0 < nf; f0 += bt) {
        const int Fb = std::min(bt, nf - f0);
        ReducedBatch rb;
        fsi_status s = reduced_solve_batch(k, reinterpret_cast<const double2*>(KR), reinterpret_cast<const double2*>(DR),
                                           reinterpret_cast<const double2*>(MR), reinterpret_cast<const double2*>(fR),
                                           nrhs, f_hz + f0, Fb, ws, red, rb, st);
        if (s != FSI_OK) return s;
        const dim3 grid(cdiv(n, 256), Fb);
        const double2* Vd = reinterpret_cast<const double2*>(V);
        if (nrhs == 1)
            backproject_kernel<1><<<grid, 256, 0, st>>>(Vd, n, k, rb.G, rb.cs, nrhs, x);
        else if (nrhs == 2)
            backproject_kernel<2><<<grid, 256, 0, st>>>(Vd, n, k, rb.G, rb.cs, nrhs, x);
        else if (nrhs <= 4)
            backproject_kernel<4><<<grid, 256, 0, st>>>(Vd, n, k, rb.G, rb.cs, nrhs, x);
        else
            backproject_kernel<8><<<grid, 256, 0, st>>>(Vd, n, k, rb.G, rb.cs, nrhs, x);
        ROM_LAUNCH();
        ROM_CUDA(cudaMemsetAsync(norms, 0, sizeof(double) * Fb * nrhs, st));
        launch_residual(m, rb.omega, 0.0, Fb, x, int64_t(nrhs) * n, Fd, nrhs, r, int64_t(nrhs) * n, norms, false,
                        st);
        ROM_LAUNCH();
        ROM_CUDA(cudaMemcpyAsync(hn.data(), norms, sizeof(double) * Fb * nrhs, cudaMemcpyDeviceToHost, st));
        ROM_CUDA(cudaStreamSynchronize(st));
        for (int q = 0; q < Fb * nrhs; ++q) {
            const double d = hfn[q % nrhs];
            relres[int64_t(f0) * nrhs + q] = d > 0 ? std::sqrt(hn[q] / d) : 0.0;
        }
    }
    return FSI_OK;
}

}  // extern "C"
