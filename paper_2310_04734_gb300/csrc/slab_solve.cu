// Forward and backward substitution with the stored block-banded factor (paper
// Sec. 2: the direct solve of A(w) x = f behind each frequency step).
//
// Stored per slab k and frequency: the factor rows [L11\U_kk | U_k,k+1 | U_k,k+2]
// (b x 3b, row major), the multipliers L21 of the next slab's rows (b x b) and the
// row permutation of the stacked pair [slab k; slab k+1] (2b entries).
//
//   forward,  k = 0..nz-1:  t = P_k [y_k; y_k+1],  y_k = L11^-1 t_top,
//                           y_k+1 = t_bot - L21 y_k
//   backward, k = nz-1..0:  v = y_k - U_k,k+1 y_k+1 - U_k,k+2 y_k+2,  y_k = U_kk^-1 v
//
// Each slab step is two launches.  The dense rectangular products (L21: b x b,
// [U_k,k+1 U_k,k+2]: b x 2b -- three quarters of the factor's bytes) are
// matrix-vector kernels over (row tiles x frequencies), so every SM streams
// factor rows.  The triangles are solved one CTA per frequency by left-looking
// blocked substitution: for each 32-row block, 16 warps form the dot products of
// the block's rows with the solved part (two rows per warp, eight 16-byte loads
// in flight per row and lane), then one warp per right-hand side substitutes
// through the 32 x 32 diagonal triangle staged in shared memory.  The diagonal
// solve is true substitution: multiplying by explicit inverses of the diagonal
// blocks degrades the FP32 factor as a preconditioner (x = T^-1 v cancels).
#include <algorithm>

#include "kernels.cuh"
#include "prof.h"

namespace fsi {

namespace {

constexpr int kTriThreads = 512;   // 16 warps x 2 rows = one 32-row block
constexpr int kTB = 32;            // diagonal block size
constexpr int kTS = kTB + 1;       // staged diagonal block stride
constexpr int kQ = 8;              // 16-byte loads per row and lane kept in flight
constexpr int kGvWarps = 8;        // matrix-vector kernel: warps per CTA
constexpr int kGvRows = 4;         // rows per warp
constexpr int kMaxNR = 4;          // right-hand sides per launch
constexpr size_t kMaxSolveSmem = 220 * 1024;

// 16-byte load unit: two FP32 complex entries (VEC) or one entry.
template <typename T2, bool VEC>
struct Ld;
template <>
struct Ld<float2, true> {
    using V = float4;
    static constexpr int E = 2;
};
template <>
struct Ld<float2, false> {
    using V = float2;
    static constexpr int E = 1;
};
template <bool VEC>
struct Ld<double2, VEC> {
    using V = double2;
    static constexpr int E = 1;
};

// acc += m . x over the E complex entries of one load unit
__device__ __forceinline__ void vfma(float2& acc, float4 m, float4 x) {
    acc.x = fmaf(m.x, x.x, acc.x);
    acc.x = fmaf(-m.y, x.y, acc.x);
    acc.y = fmaf(m.x, x.y, acc.y);
    acc.y = fmaf(m.y, x.x, acc.y);
    acc.x = fmaf(m.z, x.z, acc.x);
    acc.x = fmaf(-m.w, x.w, acc.x);
    acc.y = fmaf(m.z, x.w, acc.y);
    acc.y = fmaf(m.w, x.z, acc.y);
}
__device__ __forceinline__ void vfma(float2& acc, float2 m, float2 x) { cfma(acc, m, x); }
__device__ __forceinline__ void vfma(double2& acc, double2 m, double2 x) { cfma(acc, m, x); }

template <typename V>
__device__ __forceinline__ V vzero() {
    return V{};
}

template <typename T2, int N>
__device__ __forceinline__ void warp_sum(T2 (&a)[N]) {
#pragma unroll
    for (int c = 0; c < N; ++c)
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            a[c].x += __shfl_xor_sync(0xffffffffu, a[c].x, off);
            a[c].y += __shfl_xor_sync(0xffffffffu, a[c].y, off);
        }
}

// Lane partials of  a0[c] += row0[j] t[c*ts + j],  a1[c] += row1[j] t[c*ts + j]  for j in [j0, j1)
// (j0, j1 multiples of E; row1 may be null).  Loads of kQ units per row are issued before use.
template <typename T2, bool VEC, int NR>
__device__ __forceinline__ void row_dot2(const T2* __restrict__ row0, const T2* __restrict__ row1, const T2* t,
                                         int ts, int j0, int j1, T2 (&a0)[NR], T2 (&a1)[NR]) {
    using V = typename Ld<T2, VEC>::V;
    constexpr int E = Ld<T2, VEC>::E;
    const int lane = threadIdx.x & 31;
    for (int jb = j0 + lane * E; jb < j1; jb += 32 * E * kQ) {
        V m0[kQ], m1[kQ];
#pragma unroll
        for (int q = 0; q < kQ; ++q) {
            const int j = jb + q * 32 * E;
            m0[q] = j < j1 ? __ldg(reinterpret_cast<const V*>(row0 + j)) : vzero<V>();
            m1[q] = (row1 && j < j1) ? __ldg(reinterpret_cast<const V*>(row1 + j)) : vzero<V>();
        }
#pragma unroll
        for (int q = 0; q < kQ; ++q) {
            const int j = jb + q * 32 * E;
            if (j < j1) {
#pragma unroll
                for (int c = 0; c < NR; ++c) {
                    const V xv = *reinterpret_cast<const V*>(t + c * ts + j);
                    vfma(a0[c], m0[q], xv);
                    vfma(a1[c], m1[q], xv);
                }
            }
        }
    }
}

// One warp: v[0..nb) <- T^-1 v for the nb x nb triangle staged in D (stride kTS).
// LOWER: unit lower (forward); else upper with its diagonal (backward).
template <typename T2, bool LOWER>
__device__ __forceinline__ void tri32(const T2* D, int nb, T2* v) {
    using R = decltype(T2::x);
    const int lane = threadIdx.x & 31;
    T2 x = lane < nb ? v[lane] : mk<T2>(R(0), R(0));
    if (LOWER) {
        for (int jj = 0; jj < nb; ++jj) {
            T2 xj;
            xj.x = __shfl_sync(0xffffffffu, x.x, jj);
            xj.y = __shfl_sync(0xffffffffu, x.y, jj);
            if (lane > jj && lane < nb) cfms(x, D[lane * kTS + jj], xj);
        }
    } else {
        const T2 dinv = lane < nb ? cinv(D[lane * kTS + lane]) : mk<T2>(R(0), R(0));
        for (int jj = nb - 1; jj >= 0; --jj) {
            if (lane == jj) x = cmul(x, dinv);
            T2 xj;
            xj.x = __shfl_sync(0xffffffffu, x.x, jj);
            xj.y = __shfl_sync(0xffffffffu, x.y, jj);
            if (lane < jj) cfms(x, D[lane * kTS + jj], xj);
        }
    }
    if (lane < nb) v[lane] = x;
}

// Rows r0 = bs + warp and r1 = r0 + 16 of a block: stage their diagonal-block entries,
// subtract their dot products with the solved columns [j0, j1) of t.
template <typename T2, bool VEC, int NR>
__device__ __forceinline__ void block_rows(const T2* __restrict__ Uk, int ld, int bs, int nb, int j0, int j1, T2* t,
                                           int ts, T2* D) {
    using R = decltype(T2::x);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int r0 = bs + warp, r1 = bs + warp + 16;
    const bool h0 = r0 < bs + nb, h1 = r1 < bs + nb;
    const T2 z = mk<T2>(R(0), R(0));
    const T2 d0 = (h0 && lane < nb) ? Uk[int64_t(r0) * ld + bs + lane] : z;
    const T2 d1 = (h1 && lane < nb) ? Uk[int64_t(r1) * ld + bs + lane] : z;
    if (j1 > j0 && h0) {
        T2 a0[NR], a1[NR];
#pragma unroll
        for (int c = 0; c < NR; ++c) a0[c] = a1[c] = z;
        row_dot2<T2, VEC, NR>(Uk + int64_t(r0) * ld, h1 ? Uk + int64_t(r1) * ld : nullptr, t, ts, j0, j1, a0, a1);
        warp_sum(a0);
        warp_sum(a1);
        if (lane == 0) {
#pragma unroll
            for (int c = 0; c < NR; ++c) {
                t[c * ts + r0] = csub(t[c * ts + r0], a0[c]);
                if (h1) t[c * ts + r1] = csub(t[c * ts + r1], a1[c]);
            }
        }
    }
    if (h0) D[(r0 - bs) * kTS + lane] = d0;
    if (h1) D[(r1 - bs) * kTS + lane] = d1;
}

// Forward triangle of slab k, one CTA per frequency.  y points at slab k of the
// frequency-0 vector (right-hand side c at offset c*n); m = 2b, or b on the last slab.
template <typename T2, bool VEC, int NR>
__global__ void __launch_bounds__(kTriThreads) tri_fwd_kernel(const T2* __restrict__ U, int64_t sU,
                                                              const int32_t* __restrict__ perm, int64_t sPerm,
                                                              T2* y, int64_t sY, int64_t n, int b, int m,
                                                              const int32_t* __restrict__ flist) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T2* t = reinterpret_cast<T2*>(smem_raw);   // [NR][m]
    T2* D = t + size_t(NR) * m;                // [kTB][kTS]
    const int f = flist ? flist[blockIdx.x] : blockIdx.x, warp = threadIdx.x >> 5;
    const T2* Uk = U + f * sU;
    const int32_t* pk = perm + f * sPerm;
    T2* yf = y + f * sY + int64_t(blockIdx.y) * NR * n;   // this CTA's right-hand sides
    for (int idx = threadIdx.x; idx < m * NR; idx += blockDim.x) {
        const int c = idx / m, i = idx - c * m;
        t[c * m + i] = yf[c * n + pk[i]];
    }
    __syncthreads();
    for (int bs = 0; bs < b; bs += kTB) {
        const int nb = min(kTB, b - bs);
        block_rows<T2, VEC, NR>(Uk, 3 * b, bs, nb, 0, bs, t, m, D);
        __syncthreads();
        if (warp < NR) tri32<T2, true>(D, nb, t + warp * m + bs);
        __syncthreads();
    }
    for (int idx = threadIdx.x; idx < m * NR; idx += blockDim.x) {
        const int c = idx / m, i = idx - c * m;
        yf[c * n + i] = t[c * m + i];
    }
}

// Backward triangle of slab k (after the far columns were subtracted), one CTA per frequency.
template <typename T2, bool VEC, int NR>
__global__ void __launch_bounds__(kTriThreads) tri_bwd_kernel(const T2* __restrict__ U, int64_t sU, T2* y,
                                                              int64_t sY, int64_t n, int b,
                                                              const int32_t* __restrict__ flist) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T2* v = reinterpret_cast<T2*>(smem_raw);   // [NR][b]
    T2* D = v + size_t(NR) * b;                // [kTB][kTS]
    const int f = flist ? flist[blockIdx.x] : blockIdx.x, warp = threadIdx.x >> 5;
    const T2* Uk = U + f * sU;
    T2* yf = y + f * sY + int64_t(blockIdx.y) * NR * n;   // this CTA's right-hand sides
    for (int idx = threadIdx.x; idx < b * NR; idx += blockDim.x) {
        const int c = idx / b, i = idx - c * b;
        v[c * b + i] = yf[c * n + i];
    }
    __syncthreads();
    for (int blk = (b + kTB - 1) / kTB - 1; blk >= 0; --blk) {
        const int bs = blk * kTB, nb = min(kTB, b - bs);
        block_rows<T2, VEC, NR>(Uk, 3 * b, bs, nb, bs + nb, b, v, b, D);
        __syncthreads();
        if (warp < NR) tri32<T2, false>(D, nb, v + warp * b + bs);
        __syncthreads();
    }
    for (int idx = threadIdx.x; idx < b * NR; idx += blockDim.x) {
        const int c = idx / b, i = idx - c * b;
        yf[c * n + i] = v[c * b + i];
    }
}

// out[c*n + i] -= sum_j M[i*ldm + j] x[c*n + j]  for i < rows, j < cols; frequency f = blockIdx.y.
// Each warp holds kGvRows rows; x is read once per column chunk and reused across them.
template <typename T2, bool VEC, int NR>
__global__ void __launch_bounds__(kGvWarps * 32, 2) slab_gemv_kernel(const T2* __restrict__ M, int64_t sM, int ldm,
                                                                  int rows, int cols, const T2* x, int64_t sX,
                                                                  T2* out, int64_t sO, int64_t n,
                                                                  const int32_t* __restrict__ flist) {
    using R = decltype(T2::x);
    using V = typename Ld<T2, VEC>::V;
    constexpr int E = Ld<T2, VEC>::E;
    constexpr int U2 = 2;   // column chunks per iteration
    const int f = flist ? flist[blockIdx.y] : blockIdx.y;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int row0 = (blockIdx.x * kGvWarps + warp) * kGvRows;
    if (row0 >= rows) return;
    const T2* Mf = M + f * sM;
    const T2* xf = x + f * sX;
    T2* of = out + f * sO;
    T2 acc[kGvRows][NR];
#pragma unroll
    for (int r = 0; r < kGvRows; ++r)
#pragma unroll
        for (int c = 0; c < NR; ++c) acc[r][c] = mk<T2>(R(0), R(0));
    const T2* mrow[kGvRows];
#pragma unroll
    for (int r = 0; r < kGvRows; ++r) mrow[r] = Mf + int64_t(min(row0 + r, rows - 1)) * ldm;
    for (int jb = lane * E; jb < cols; jb += 32 * E * U2) {
        V mv[U2][kGvRows], xv[U2][NR];
#pragma unroll
        for (int u = 0; u < U2; ++u) {
            const int j = jb + u * 32 * E;
            const bool in = j < cols;
#pragma unroll
            for (int r = 0; r < kGvRows; ++r)
                mv[u][r] = (in && row0 + r < rows) ? __ldg(reinterpret_cast<const V*>(mrow[r] + j)) : vzero<V>();
#pragma unroll
            for (int c = 0; c < NR; ++c)
                xv[u][c] = in ? __ldg(reinterpret_cast<const V*>(xf + c * n + j)) : vzero<V>();
        }
#pragma unroll
        for (int u = 0; u < U2; ++u)
#pragma unroll
            for (int r = 0; r < kGvRows; ++r)
#pragma unroll
                for (int c = 0; c < NR; ++c) vfma(acc[r][c], mv[u][r], xv[u][c]);
    }
#pragma unroll
    for (int r = 0; r < kGvRows; ++r) warp_sum(acc[r]);
    if (lane == 0) {
#pragma unroll
        for (int r = 0; r < kGvRows; ++r)
            if (row0 + r < rows)
#pragma unroll
                for (int c = 0; c < NR; ++c) {
                    T2& o = of[c * n + row0 + r];
                    o = csub(o, acc[r][c]);
                }
    }
}

template <typename T2, bool VEC, int NR>
void tri_fwd(const T2* U, int64_t sU, const int32_t* perm, int64_t sPerm, T2* y, int64_t sY, int64_t n, int b, int m,
             dim3 grid, const int32_t* flist, size_t smem, cudaStream_t st) {
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(tri_fwd_kernel<T2, VEC, NR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             int(kMaxSolveSmem));
        attr = true;
    }
    tri_fwd_kernel<T2, VEC, NR><<<grid, kTriThreads, smem, st>>>(U, sU, perm, sPerm, y, sY, n, b, m, flist);
}

template <typename T2, bool VEC, int NR>
void tri_bwd(const T2* U, int64_t sU, T2* y, int64_t sY, int64_t n, int b, dim3 grid, const int32_t* flist,
             size_t smem, cudaStream_t st) {
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(tri_bwd_kernel<T2, VEC, NR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             int(kMaxSolveSmem));
        attr = true;
    }
    tri_bwd_kernel<T2, VEC, NR><<<grid, kTriThreads, smem, st>>>(U, sU, y, sY, n, b, flist);
}

template <typename T2, bool VEC, int NR>
void gemv(const T2* M, int64_t sM, int ldm, int rows, int cols, const T2* x, int64_t sX, T2* out, int64_t sO,
          int64_t n, int F, const int32_t* flist, cudaStream_t st) {
    const int per = kGvWarps * kGvRows;
    dim3 grid((rows + per - 1) / per, F);
    slab_gemv_kernel<T2, VEC, NR><<<grid, kGvWarps * 32, 0, st>>>(M, sM, ldm, rows, cols, x, sX, out, sO, n, flist);
}

// Right-hand sides per triangle CTA.  The triangle of one frequency is a chain of
// dependent block steps on one SM, issue-bound on its FMAs, so the right-hand sides
// are spread over CTAs (each rereads the triangle, mostly from L2) while the grid
// still fits on the SMs at once.
int tri_rhs_per_cta(int F, int nc) {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    for (int nr : {1, 2, 4})
        if (nc % nr == 0 && int64_t(F) * (nc / nr) <= sms) return nr;
    return nc % 4 == 0 ? 4 : (nc % 2 == 0 ? 2 : 1);
}

// Right-hand sides per launch such that the triangle's vectors fit in shared memory.
template <typename T2>
int rhs_per_launch(int rows) {
    const size_t dbytes = size_t(kTB) * kTS * sizeof(T2);
    const size_t per = size_t(rows) * sizeof(T2);
    const int fit = int((kMaxSolveSmem - dbytes) / per);
    return std::max(1, std::min(kMaxNR, fit));
}

template <typename T2, bool VEC>
void fwd_slab(const T2* U, const T2* L, int64_t sU, int64_t sL, const int32_t* perm, int64_t sPerm, T2* y,
              int64_t sY, int64_t n, int b, int k, int nz, int nrhs, int F, const int32_t* flist, cudaStream_t st) {
    const int m = (k + 1 < nz) ? 2 * b : b;
    const int step = rhs_per_launch<T2>(m);
    for (int c0 = 0; c0 < nrhs; c0 += step) {
        const int nc = std::min(step, nrhs - c0);
        T2* yk = y + int64_t(c0) * n + int64_t(k) * b;
        {
            const int nr = tri_rhs_per_cta(F, nc);
            const dim3 grid(unsigned(F), unsigned(nc / nr));
            const size_t smem = (size_t(nr) * m + size_t(kTB) * kTS) * sizeof(T2);
            ProfScope ps(PK_SOLVE, 8.0 * F * nc * double(b) * b / 2.0, st);
            switch (nr) {
                case 1: tri_fwd<T2, VEC, 1>(U, sU, perm, sPerm, yk, sY, n, b, m, grid, flist, smem, st); break;
                case 2: tri_fwd<T2, VEC, 2>(U, sU, perm, sPerm, yk, sY, n, b, m, grid, flist, smem, st); break;
                default: tri_fwd<T2, VEC, 4>(U, sU, perm, sPerm, yk, sY, n, b, m, grid, flist, smem, st); break;
            }
        }
        if (m == 2 * b) {
            ProfScope ps(PK_GEMV, 8.0 * F * nc * double(b) * b, st);
            switch (nc) {
                case 1: gemv<T2, VEC, 1>(L, sL, b, b, b, yk, sY, yk + b, sY, n, F, flist, st); break;
                case 2: gemv<T2, VEC, 2>(L, sL, b, b, b, yk, sY, yk + b, sY, n, F, flist, st); break;
                case 3: gemv<T2, VEC, 3>(L, sL, b, b, b, yk, sY, yk + b, sY, n, F, flist, st); break;
                default: gemv<T2, VEC, 4>(L, sL, b, b, b, yk, sY, yk + b, sY, n, F, flist, st); break;
            }
        }
    }
}

template <typename T2, bool VEC>
void bwd_slab(const T2* U, int64_t sU, T2* y, int64_t sY, int64_t n, int b, int k, int nz, int nrhs, int F,
              const int32_t* flist, cudaStream_t st) {
    const int far = std::min(2, nz - 1 - k) * b;
    const int step = rhs_per_launch<T2>(b);
    for (int c0 = 0; c0 < nrhs; c0 += step) {
        const int nc = std::min(step, nrhs - c0);
        T2* yk = y + int64_t(c0) * n + int64_t(k) * b;
        if (far > 0) {
            ProfScope ps(PK_GEMV, 8.0 * F * nc * double(far) * b, st);
            switch (nc) {
                case 1: gemv<T2, VEC, 1>(U + b, sU, 3 * b, b, far, yk + b, sY, yk, sY, n, F, flist, st); break;
                case 2: gemv<T2, VEC, 2>(U + b, sU, 3 * b, b, far, yk + b, sY, yk, sY, n, F, flist, st); break;
                case 3: gemv<T2, VEC, 3>(U + b, sU, 3 * b, b, far, yk + b, sY, yk, sY, n, F, flist, st); break;
                default: gemv<T2, VEC, 4>(U + b, sU, 3 * b, b, far, yk + b, sY, yk, sY, n, F, flist, st); break;
            }
        }
        const int nr = tri_rhs_per_cta(F, nc);
        const dim3 grid(unsigned(F), unsigned(nc / nr));
        const size_t smem = (size_t(nr) * b + size_t(kTB) * kTS) * sizeof(T2);
        ProfScope ps(PK_SOLVE, 8.0 * F * nc * double(b) * b / 2.0, st);
        switch (nr) {
            case 1: tri_bwd<T2, VEC, 1>(U, sU, yk, sY, n, b, grid, flist, smem, st); break;
            case 2: tri_bwd<T2, VEC, 2>(U, sU, yk, sY, n, b, grid, flist, smem, st); break;
            default: tri_bwd<T2, VEC, 4>(U, sU, yk, sY, n, b, grid, flist, smem, st); break;
        }
    }
}

// Two-entry FP32 loads need every row start and vector offset even (b even) and
// 16-byte aligned base pointers.
template <typename T2>
bool vec_ok(int b, const void* a, const void* c, const void* d) {
    if (sizeof(T2) != 8) return false;
    auto al = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; };
    return (b % 2 == 0) && al(a) && al(c) && al(d);
}

}  // namespace

template <typename R>
void launch_slab_solve_fwd(const typename Cplx<R>::T* U, const typename Cplx<R>::T* L, int64_t sU, int64_t sL,
                           const int32_t* perm, int64_t sPerm, typename Cplx<R>::T* y, int64_t sY, int64_t n, int b,
                           int k, int nz, int nrhs, int F, const int32_t* flist, cudaStream_t st) {
    using T2 = typename Cplx<R>::T;
    const bool strides_even = (sU % 2 == 0) && (sL % 2 == 0) && (sY % 2 == 0) && (n % 2 == 0);
    if (strides_even && vec_ok<T2>(b, U, L, y))
        fwd_slab<T2, true>(U, L, sU, sL, perm, sPerm, y, sY, n, b, k, nz, nrhs, F, flist, st);
    else
        fwd_slab<T2, false>(U, L, sU, sL, perm, sPerm, y, sY, n, b, k, nz, nrhs, F, flist, st);
}

template <typename R>
void launch_slab_solve_bwd(const typename Cplx<R>::T* U, int64_t sU, typename Cplx<R>::T* y, int64_t sY, int64_t n,
                           int b, int k, int nz, int nrhs, int F, const int32_t* flist, cudaStream_t st) {
    using T2 = typename Cplx<R>::T;
    const bool strides_even = (sU % 2 == 0) && (sY % 2 == 0) && (n % 2 == 0);
    if (strides_even && vec_ok<T2>(b, U, y, y))
        bwd_slab<T2, true>(U, sU, y, sY, n, b, k, nz, nrhs, F, flist, st);
    else
        bwd_slab<T2, false>(U, sU, y, sY, n, b, k, nz, nrhs, F, flist, st);
}

#define FSI_SOLVE_INSTANTIATE(R)                                                                                    \
    template void launch_slab_solve_fwd<R>(const Cplx<R>::T*, const Cplx<R>::T*, int64_t, int64_t, const int32_t*, \
                                           int64_t, Cplx<R>::T*, int64_t, int64_t, int, int, int, int, int,         \
                                           const int32_t*, cudaStream_t);                                           \
    template void launch_slab_solve_bwd<R>(const Cplx<R>::T*, int64_t, Cplx<R>::T*, int64_t, int64_t, int, int,    \
                                           int, int, int, const int32_t*, cudaStream_t);

FSI_SOLVE_INSTANTIATE(float)
FSI_SOLVE_INSTANTIATE(double)

}  // namespace fsi
