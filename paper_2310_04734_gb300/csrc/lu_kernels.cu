// Batched dense kernels of the block-banded LU (paper Sec. 2: one direct solve
// of A(w) per frequency step; here the slab-ordered matrix is factored as a
// band whose pivot search spans the stacked panel of two consecutive slabs).
//
// Matrices are row-major complex (float2 / double2), batched over frequencies
// with a fixed element stride.  The factorisation of one stacked window is a
// right-looking partial LU over its first b columns:
//   for each outer panel J (width NB):
//     for each sub-panel j in J (width nbw, held in shared memory):
//       panel LU with partial pivoting, row swaps inside the outer panel,
//       unit-lower TRSM and a GEMM update restricted to the outer panel
//     row swaps outside the outer panel, TRSM of the NB pivot rows, and the
//     trailing GEMM update with K = NB.
#include <cfloat>
#include <cmath>

#include "kernels.cuh"
#include "prof.h"

namespace fsi {

namespace {

constexpr int kPanelThreads = 1024;
constexpr size_t kMaxPanelSmem = 226 * 1024;

template <typename T2>
struct Real;
template <>
struct Real<float2> {
    using R = float;
};
template <>
struct Real<double2> {
    using R = double;
};

// ----------------------------------------------------------------- form rows
template <typename T2>
__global__ void form_rows_kernel(DevModel m, T2* G, int64_t sG, int ld, const double* omega, int row_slab,
                                 int g_row0, int col_slab0, int wcols) {
    using R = typename Real<T2>::R;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int r = blockIdx.x * (blockDim.x >> 5) + warp;
    if (r >= m.b) return;
    const int f = blockIdx.y;
    const double w = omega[f];
    const int64_t grow = int64_t(row_slab) * m.b + r;
    T2* out = G + f * sG + int64_t(g_row0 + r) * ld;
    for (int c = lane; c < wcols; c += 32) out[c] = mk<T2>(R(0), R(0));
    __syncwarp();
    const double rs = row_scale(m, grow, w);
    const int64_t c0 = int64_t(col_slab0) * m.b;
    const int e1 = m.rowptr[grow + 1];
    for (int e = m.rowptr[grow] + lane; e < e1; e += 32) {
        const int64_t col = m.col[e];
        const int64_t lc = col - c0;
        if (lc < 0 || lc >= wcols) continue;
        const double2 a = a_entry(m, e, w);
        const double s = rs * col_scale(m, col, w);
        out[lc] = mk<T2>(R(a.x * s), R(a.y * s));
    }
}

// ----------------------------------------------------------------- panel LU
// (v, k, r): a candidate pivot's |.|^2, its logical row and its physical row in shared memory;
// the larger v wins, ties go to the smaller logical row (the first maximum, as in LAPACK)
template <typename R>
__device__ __forceinline__ void amax_merge(R& v, int& k, int& r, R ov, int ok, int orow) {
    if (ov > v || (ov == v && ok < k)) {
        v = ov;
        k = ok;
        r = orow;
    }
}

// butterfly: every lane ends with the warp's maximum
template <typename R>
__device__ __forceinline__ void warp_amax(R& v, int& k, int& r) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const R ov = __shfl_xor_sync(0xffffffffu, v, off);
        const int ok = __shfl_xor_sync(0xffffffffu, k, off);
        const int orow = __shfl_xor_sync(0xffffffffu, r, off);
        amax_merge(v, k, r, ov, ok, orow);
    }
}

constexpr int kPanelHdr = 2048;   // warp maxima (two slots), moved-row list and its count

// LU with partial pivoting of the panel rows [j0, m) x columns [j0, j0 + nbw), held in shared
// memory (column-major, P[t * ms + i] for physical row i).  Rows are not moved while the panel
// is factored: pos[i] is the logical position of physical row i, and the interchange of step t
// (logical rows t and q, q the pivot's position) only exchanges two entries of pos.  The rows
// still below the pivots (pos >= t) take their multipliers and rank-1 updates in place, and the
// same pass forms the argmax of column t + 1, so one barrier separates two steps.  The panel is
// written back in logical order, ipiv holds LAPACK's sequence of interchanges, and the rows that
// moved are moved in the columns [c0, j0) and [j0 + nbw, c1) as well (the rest of the outer panel).
// NBW > 0 fixes the width at compile time (index arithmetic by shifts, unrolled column loops: the
// kernel is bound by instruction issue); NBW = 0 takes it from nbw_arg.
template <typename T2, int NBW>
__global__ void __launch_bounds__(kPanelThreads) panel_kernel(T2* G, int64_t sG, int ld, int m, int j0, int nbw_arg,
                                                              int32_t* ipiv, int64_t sP, int32_t* status, int c0,
                                                              int c1) {
    const int nbw = NBW > 0 ? NBW : nbw_arg;
    using R = typename Real<T2>::R;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R* pv = reinterpret_cast<R*>(smem_raw);                            // [2][32]
    int* pk = reinterpret_cast<int*>(smem_raw + 64 * sizeof(double));  // [2][32] logical rows
    int* pr = pk + 64;                                                 // [2][32] physical rows
    int* nmoved = pr + 64;
    int* moved = nmoved + 4;                                           // physical rows whose pos changed
    const int mr = m - j0;
    int* pos = reinterpret_cast<int*>(smem_raw + kPanelHdr);
    T2* P = reinterpret_cast<T2*>(smem_raw + kPanelHdr + ((size_t(mr) * 4 + 15) & ~size_t(15)));
    const int f = blockIdx.x;
    T2* A = G + f * sG;
    const int ms = mr | 1;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    for (int idx = tid; idx < mr * nbw; idx += blockDim.x) {
        const int i = idx / nbw, t = idx - i * nbw;
        P[t * ms + i] = A[int64_t(j0 + i) * ld + j0 + t];
    }
    for (int i = tid; i < mr; i += blockDim.x) pos[i] = i;
    if (tid == 0) *nmoved = 0;
    __syncthreads();
    R bv = R(-1);
    int bk = 0x7fffffff, br = -1;
    for (int i = tid; i < mr; i += blockDim.x) {
        const T2 v = P[i];
        amax_merge(bv, bk, br, v.x * v.x + v.y * v.y, i, i);
    }
    // with the width fixed at compile time every step is unrolled, so each step's column loop has
    // its own trip count (no predicated-off columns)
#pragma unroll(NBW > 0 ? NBW : 1)
    for (int t = 0; t < nbw; ++t) {
        warp_amax(bv, bk, br);
        const int slot = (t & 1) * 32;
        if (lane == 0) {
            pv[slot + warp] = bv;
            pk[slot + warp] = bk;
            pr[slot + warp] = br;
        }
        __syncthreads();
        bv = lane < nw ? pv[slot + lane] : R(-1);
        bk = lane < nw ? pk[slot + lane] : 0x7fffffff;
        br = lane < nw ? pr[slot + lane] : -1;
        warp_amax(bv, bk, br);
        const int q = bk, p = br;
        const bool bad = !(bv > R(0)) || isinf(bv) || p < 0;
        R nv = R(-1);
        int nk = 0x7fffffff, nr = -1;   // argmax of column t + 1 over the rows left below
        const bool next = t + 1 < nbw;
        if (bad) {
            // no usable pivot: the row at position t stays there and the column is left as it is
            if (tid == 0) {
                status[f] = 1;
                ipiv[f * sP + j0 + t] = j0 + t;
            }
            for (int i = tid; i < mr && next; i += blockDim.x) {
                const int ps = pos[i];
                if (ps <= t) continue;
                const T2 v = P[(t + 1) * ms + i];
                amax_merge(nv, nk, nr, v.x * v.x + v.y * v.y, ps, i);
            }
        } else {
            const T2 inv = cinv(P[t * ms + p]);
            if (tid == 0) ipiv[f * sP + j0 + t] = j0 + q;
            for (int i = tid; i < mr; i += blockDim.x) {
                int ps = pos[i];
                if (i == p) {
                    pos[i] = t;
                    continue;
                }
                if (ps < t) continue;   // a pivot row of an earlier step
                if (ps == t) {          // displaced by the interchange
                    ps = q;
                    pos[i] = q;
                }
                const T2 l = cmul(P[t * ms + i], inv);
                P[t * ms + i] = l;
                if constexpr (NBW > 0) {
#pragma unroll
                    for (int u = 1; u < NBW; ++u)
                        if (u > t) cfms(P[u * ms + i], l, P[u * ms + p]);
                } else {
                    for (int u = t + 1; u < nbw; ++u) cfms(P[u * ms + i], l, P[u * ms + p]);
                }
                if (next) {
                    const T2 v = P[(t + 1) * ms + i];
                    amax_merge(nv, nk, nr, v.x * v.x + v.y * v.y, ps, i);
                }
            }
        }
        bv = nv;
        bk = nk;
        br = nr;
    }
    __syncthreads();
    for (int idx = tid; idx < mr * nbw; idx += blockDim.x) {
        const int i = idx / nbw, t = idx - i * nbw;
        A[int64_t(j0 + pos[i]) * ld + j0 + t] = P[t * ms + i];
    }
    for (int i = tid; i < mr; i += blockDim.x)
        if (pos[i] != i) moved[atomicAdd(nmoved, 1)] = i;
    // the same interchanges in the other columns of the outer panel, staged through shared memory
    // nbw columns at a time (the moved rows are at most mr, so a chunk fits in the panel's space)
    const int nleft = j0 - c0, nother = nleft + max(c1 - j0 - nbw, 0);
    __syncthreads();
    const int nm = *nmoved;
    for (int cb = 0; cb < nother && nm > 0; cb += nbw) {
        for (int e = tid; e < nm * nbw; e += blockDim.x) {
            const int k = e / nbw, c = cb + e - k * nbw;
            if (c >= nother) continue;
            const int col = c < nleft ? c0 + c : j0 + nbw + (c - nleft);
            P[e] = A[int64_t(j0 + moved[k]) * ld + col];
        }
        __syncthreads();
        for (int e = tid; e < nm * nbw; e += blockDim.x) {
            const int k = e / nbw, c = cb + e - k * nbw;
            if (c >= nother) continue;
            const int col = c < nleft ? c0 + c : j0 + nbw + (c - nleft);
            A[int64_t(j0 + pos[moved[k]]) * ld + col] = P[e];
        }
        __syncthreads();
    }
}

// ----------------------------------------------------------------- laswp
constexpr int kSwpCols = 32;      // columns per CTA
constexpr int kSwpThreads = 256;

// Row interchanges ipiv[j .. j + cnt) (LAPACK order) applied to the columns [a0, a1) and [b0, b1).
// Each CTA forms the composite permutation of the rows involved (every involved row is traced
// back through the interchanges by one thread), stages its columns of the rows that move in
// shared memory and writes them to their destinations: two passes of coalesced row segments in
// place of cnt dependent swaps per column.
template <typename T2>
__global__ void __launch_bounds__(kSwpThreads) laswp_kernel(T2* G, int64_t sG, int ld, int j, int cnt,
                                                            const int32_t* ipiv, int64_t sP, int a0, int a1, int b0,
                                                            int b1) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    int* piv = reinterpret_cast<int*>(smem_raw);   // [cnt]
    int* src = piv + cnt;                          // [2 cnt]
    int* dst = src + 2 * cnt;                      // [2 cnt]
    int* nmv = dst + 2 * cnt;
    T2* S = reinterpret_cast<T2*>(smem_raw + ((size_t(5 * cnt + 4) * 4 + 15) & ~size_t(15)));   // [2 cnt][kSwpCols]
    const int f = blockIdx.y, tid = threadIdx.x;
    T2* A = G + f * sG;
    for (int t = tid; t < cnt; t += blockDim.x) piv[t] = ipiv[f * sP + j + t];
    if (tid == 0) *nmv = 0;
    __syncthreads();
    // involved rows: j + t for t < cnt, and the first occurrence of each target below the block
    for (int e = tid; e < 2 * cnt; e += blockDim.x) {
        int r;
        if (e < cnt) {
            r = j + e;
        } else {
            const int t = e - cnt;
            r = piv[t];
            if (r < j + cnt) continue;
            bool first = true;
            for (int u = 0; u < t && first; ++u) first = piv[u] != r;
            if (!first) continue;
        }
        int s = r;   // the row whose content ends at r: the interchanges applied in reverse
        for (int t = cnt - 1; t >= 0; --t) {
            const int p = piv[t];
            if (s == j + t) s = p;
            else if (s == p) s = j + t;
        }
        if (s != r) {
            const int k = atomicAdd(nmv, 1);
            src[k] = s;
            dst[k] = r;
        }
    }
    __syncthreads();
    const int n = *nmv, na = a1 > a0 ? a1 - a0 : 0;
    const int ntot = na + (b1 > b0 ? b1 - b0 : 0);
    const int q0 = blockIdx.x * kSwpCols;
    for (int e = tid; e < n * kSwpCols; e += blockDim.x) {
        const int k = e / kSwpCols, q = q0 + e - k * kSwpCols;
        if (q >= ntot) continue;
        const int col = q < na ? a0 + q : b0 + (q - na);
        S[e] = A[int64_t(src[k]) * ld + col];
    }
    __syncthreads();
    for (int e = tid; e < n * kSwpCols; e += blockDim.x) {
        const int k = e / kSwpCols, q = q0 + e - k * kSwpCols;
        if (q >= ntot) continue;
        const int col = q < na ? a0 + q : b0 + (q - na);
        A[int64_t(dst[k]) * ld + col] = S[e];
    }
}

// ----------------------------------------------------------------- trsm (unit lower)
constexpr int kTrsmThreads = 128;
template <typename T2>
__global__ void __launch_bounds__(kTrsmThreads) trsm_kernel(T2* G, int64_t sG, int ld, int j, int cnt, int c0,
                                                            int c1) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T2* Ls = reinterpret_cast<T2*>(smem_raw);     // cnt x cnt
    T2* Bs = Ls + cnt * cnt;                      // cnt x kTrsmThreads
    const int f = blockIdx.y;
    T2* A = G + f * sG;
    for (int idx = threadIdx.x; idx < cnt * cnt; idx += blockDim.x) {
        const int r = idx / cnt, c = idx - r * cnt;
        Ls[idx] = A[int64_t(j + r) * ld + j + c];
    }
    const int c = c0 + blockIdx.x * blockDim.x + threadIdx.x;
    const bool live = c < c1;
    if (live)
        for (int i = 0; i < cnt; ++i) Bs[i * kTrsmThreads + threadIdx.x] = A[int64_t(j + i) * ld + c];
    __syncthreads();
    if (!live) return;
    for (int i = 1; i < cnt; ++i) {
        T2 acc = Bs[i * kTrsmThreads + threadIdx.x];
        for (int t = 0; t < i; ++t) cfms(acc, Ls[i * cnt + t], Bs[t * kTrsmThreads + threadIdx.x]);
        Bs[i * kTrsmThreads + threadIdx.x] = acc;
    }
    for (int i = 1; i < cnt; ++i) A[int64_t(j + i) * ld + c] = Bs[i * kTrsmThreads + threadIdx.x];
}

// Same solve for a fixed triangle size CNT: the thread's column lives in registers and the
// substitution is written column by column (b_t final, then every row below it updated), so
// the CNT - t - 1 updates of a step are independent and no shared-memory traffic touches the
// right-hand side; only the triangle (unit lower part) is staged in shared memory.
template <typename T2, int CNT>
__global__ void __launch_bounds__(kTrsmThreads) trsm_reg_kernel(T2* G, int64_t sG, int ld, int j, int c0, int c1) {
    using R = typename Real<T2>::R;
    __shared__ T2 Ls[CNT][CNT];
    const int f = blockIdx.y;
    T2* A = G + f * sG;
    for (int idx = threadIdx.x; idx < CNT * CNT; idx += blockDim.x) {
        const int r = idx / CNT, cc = idx - r * CNT;
        Ls[r][cc] = cc < r ? A[int64_t(j + r) * ld + j + cc] : mk<T2>(R(0), R(0));
    }
    __syncthreads();
    const int c = c0 + blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= c1) return;
    T2 b[CNT];
#pragma unroll
    for (int i = 0; i < CNT; ++i) b[i] = A[int64_t(j + i) * ld + c];
#pragma unroll
    for (int t = 0; t + 1 < CNT; ++t)
#pragma unroll
        for (int i = t + 1; i < CNT; ++i) cfms(b[i], Ls[i][t], b[t]);
#pragma unroll
    for (int i = 1; i < CNT; ++i) A[int64_t(j + i) * ld + c] = b[i];
}

// ----------------------------------------------------------------- gemm update
// C[r0:r1, c0:c1] -= A[r0:r1, k0:k0+K] * B[k0:k0+K, c0:c1] within one matrix of the batch
// (FP64; the FP32 update is the register-tiled kernel of cgemm_f32.cu).
constexpr int kBM = 64, kBN = 64, kBK = 16, kGemmThreads = 256;
template <typename T2>
__global__ void __launch_bounds__(kGemmThreads) gemm_update_kernel(T2* G, int64_t sG, int ld, int r0, int r1,
                                                                   int c0, int c1, int k0, int K) {
    using R = typename Real<T2>::R;
    __shared__ T2 As[kBK][kBM];
    __shared__ T2 Bs[kBK][kBN];
    const int f = blockIdx.z;
    T2* A = G + f * sG;
    const int rb = r0 + blockIdx.y * kBM, cb = c0 + blockIdx.x * kBN;
    const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
    T2 acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[i][q] = mk<T2>(R(0), R(0));
    for (int kb = 0; kb < K; kb += kBK) {
#pragma unroll
        for (int q = 0; q < (kBM * kBK) / kGemmThreads; ++q) {
            const int idx = tid + q * kGemmThreads;
            const int r = idx / kBK, kk = idx - r * kBK;
            const int gr = rb + r, gk = kb + kk;
            As[kk][r] = (gr < r1 && gk < K) ? A[int64_t(gr) * ld + k0 + gk] : mk<T2>(R(0), R(0));
        }
#pragma unroll
        for (int q = 0; q < (kBK * kBN) / kGemmThreads; ++q) {
            const int idx = tid + q * kGemmThreads;
            const int kk = idx / kBN, c = idx - kk * kBN;
            const int gc = cb + c, gk = kb + kk;
            Bs[kk][c] = (gc < c1 && gk < K) ? A[int64_t(k0 + gk) * ld + gc] : mk<T2>(R(0), R(0));
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < kBK; ++kk) {
            T2 a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int q = 0; q < 4; ++q) b[q] = Bs[kk][tx + 16 * q];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int q = 0; q < 4; ++q) cfma(acc[i][q], a[i], b[q]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int gr = rb + ty + 16 * i;
        if (gr >= r1) continue;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int gc = cb + tx + 16 * q;
            if (gc >= c1) continue;
            T2& c = A[int64_t(gr) * ld + gc];
            c = csub(c, acc[i][q]);
        }
    }
}

// ----------------------------------------------------------------- slab shift
template <typename T2>
__global__ void slab_shift_kernel(T2* G, int64_t sG, int b, int m, T2* U, int64_t sU, T2* L, int64_t sL) {
    using R = typename Real<T2>::R;
    const int f = blockIdx.y;
    const int ld = 3 * b;
    const int64_t q = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (q >= int64_t(b) * ld) return;
    const int r = int(q / ld), c = int(q - int64_t(r) * ld);
    T2* A = G + f * sG;
    U[f * sU + q] = A[q];
    const bool two = (m == 2 * b);
    if (two && c < b) L[f * sL + int64_t(r) * b + c] = A[int64_t(b + r) * ld + c];
    A[q] = (two && c < 2 * b) ? A[int64_t(b + r) * ld + b + c] : mk<T2>(R(0), R(0));
}

__global__ void perm_kernel(const int32_t* ipiv, int64_t sP, int32_t* perm, int64_t sPerm, int b, int m) {
    extern __shared__ int32_t sperm[];
    const int f = blockIdx.x;
    for (int i = threadIdx.x; i < m; i += blockDim.x) sperm[i] = i;
    __syncthreads();
    if (threadIdx.x == 0) {
        const int32_t* piv = ipiv + f * sP;
        for (int t = 0; t < b; ++t) {
            const int p = piv[t];
            const int x = sperm[t];
            sperm[t] = sperm[p];
            sperm[p] = x;
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < m; i += blockDim.x) perm[f * sPerm + i] = sperm[i];
}

// ----------------------------------------------------------------- block solves
constexpr int kSolveThreads = 1024;
constexpr int kRmax = 4;

// v <- U^-1 v for the upper n x n block (diagonal included) of `Um`.
template <typename T2>
__device__ void upper_solve(const T2* Um, int ld, int n, T2* v, int vs, int nrhs) {
    using R = typename Real<T2>::R;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const int nblk = (n + 31) / 32;
    for (int blk = nblk - 1; blk >= 0; --blk) {
        const int bs = blk * 32, be = min(bs + 32, n);
        if (be < n) {
            for (int i = bs + warp; i < be; i += nw) {
                T2 acc[kRmax];
#pragma unroll
                for (int c = 0; c < kRmax; ++c) acc[c] = mk<T2>(R(0), R(0));
                for (int jj = be + lane; jj < n; jj += 32) {
                    const T2 u = Um[int64_t(i) * ld + jj];
#pragma unroll
                    for (int c = 0; c < kRmax; ++c)
                        if (c < nrhs) cfma(acc[c], u, v[c * vs + jj]);
                }
#pragma unroll
                for (int c = 0; c < kRmax; ++c) {
                    if (c >= nrhs) break;
                    for (int off = 16; off > 0; off >>= 1) {
                        acc[c].x += __shfl_down_sync(0xffffffffu, acc[c].x, off);
                        acc[c].y += __shfl_down_sync(0xffffffffu, acc[c].y, off);
                    }
                    if (lane == 0) v[c * vs + i] = csub(v[c * vs + i], acc[c]);
                }
            }
        }
        __syncthreads();
        if (warp == 0) {
            const int i = bs + lane;
            for (int c = 0; c < nrhs; ++c) {
                T2 x = i < be ? v[c * vs + i] : mk<T2>(R(0), R(0));
                for (int ii = be - 1; ii >= bs; --ii) {
                    if (i == ii) x = cmul(x, cinv(Um[int64_t(i) * ld + i]));
                    T2 xi;
                    xi.x = __shfl_sync(0xffffffffu, x.x, ii - bs);
                    xi.y = __shfl_sync(0xffffffffu, x.y, ii - bs);
                    if (i < ii && i >= bs) cfms(x, Um[int64_t(i) * ld + ii], xi);
                }
                if (i < be) v[c * vs + i] = x;
            }
        }
        __syncthreads();
    }
}

// In-place U x = B for the upper triangle of the first n columns of each matrix;
// B is columns [c0, c0+nrhs).
template <typename T2>
__global__ void __launch_bounds__(kSolveThreads) backsub_kernel(T2* G, int64_t sG, int ld, int n, int c0,
                                                                int nrhs) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T2* v = reinterpret_cast<T2*>(smem_raw);
    T2* A = G + blockIdx.x * sG;
    for (int idx = threadIdx.x; idx < n * nrhs; idx += blockDim.x) {
        const int c = idx / n, i = idx - c * n;
        v[c * n + i] = A[int64_t(i) * ld + c0 + c];
    }
    __syncthreads();
    upper_solve(A, ld, n, v, n, nrhs);
    for (int idx = threadIdx.x; idx < n * nrhs; idx += blockDim.x) {
        const int c = idx / n, i = idx - c * n;
        A[int64_t(i) * ld + c0 + c] = v[c * n + i];
    }
}

inline unsigned ceil_div(int64_t a, int64_t b) { return unsigned((a + b - 1) / b); }

}  // namespace

// ------------------------------------------------------------------ launchers
template <typename R>
void launch_form_rows(const DevModel& m, typename Cplx<R>::T* G, int64_t sG, int ld, int F, const double* d_omega,
                      int row_slab, int g_row0, int col_slab0, int wcols, cudaStream_t st) {
    dim3 grid(ceil_div(m.b, 8), F);
    ProfScope ps(PK_FORM, 0.0, st);
    form_rows_kernel<<<grid, 256, 0, st>>>(m, G, sG, ld, d_omega, row_slab, g_row0, col_slab0, wcols);
}

// shared memory of panel_kernel for m - j0 = mr rows and width w
template <typename R>
size_t panel_smem(int mr, int w) {
    return kPanelHdr + ((size_t(mr) * 4 + 15) & ~size_t(15)) + size_t(mr | 1) * w * sizeof(typename Cplx<R>::T);
}

template <typename R>
int panel_width(int m) {
    for (int w = 32; w >= 2; w >>= 1)
        if (panel_smem<R>(m, w) <= kMaxPanelSmem) return w;
    return 1;
}

template <typename R>
static int outer_nb() {
    // FP32: K = 128 per trailing update halves the passes over the trailing matrix
    return sizeof(R) == 4 ? 128 : 32;
}

// rows of one trsm_kernel launch (its shared-memory triangle): 32 rows halve the dependent
// substitution chain of 64 and fit five CTAs per SM; the rows moved into the GEMMs that join the
// triangles cost less than that saves (measured on config 2: 18.6 vs 18.3 frequencies/s; 16 rows: 18.2)
constexpr int kTrsmMaxRows = 32;

// narrowest update (complex columns) sent to the tensor cores
constexpr int kTcMinCols = 64;

template <typename R>
void launch_panel(typename Cplx<R>::T* G, int64_t sG, int ld, int F, int m, int j0, int nbw, int32_t* ipiv,
                  int64_t sP, int32_t* status, int c0, int c1, cudaStream_t st) {
    using T2 = typename Cplx<R>::T;
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(panel_kernel<T2, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(kMaxPanelSmem));
        cudaFuncSetAttribute(panel_kernel<T2, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(kMaxPanelSmem));
        cudaFuncSetAttribute(panel_kernel<T2, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(kMaxPanelSmem));
        cudaFuncSetAttribute(panel_kernel<T2, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(kMaxPanelSmem));
        attr_set = true;
    }
    ProfScope ps(PK_PANEL, 0.0, st);
    const size_t smem = panel_smem<R>(m - j0, nbw);
    auto kern = nbw == 16 ? panel_kernel<T2, 16>
                          : nbw == 8 ? panel_kernel<T2, 8> : nbw == 32 ? panel_kernel<T2, 32> : panel_kernel<T2, 0>;
    kern<<<F, kPanelThreads, smem, st>>>(G, sG, ld, m, j0, nbw, ipiv, sP, status, c0, c1);
}

template <typename R>
void launch_laswp(typename Cplx<R>::T* G, int64_t sG, int ld, int F, int j, int cnt, const int32_t* ipiv,
                  int64_t sP, int a0, int a1, int b0, int b1, cudaStream_t st) {
    using T2 = typename Cplx<R>::T;
    const int ncols = (a1 > a0 ? a1 - a0 : 0) + (b1 > b0 ? b1 - b0 : 0);
    if (ncols <= 0 || cnt <= 0) return;
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(laswp_kernel<T2>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        attr_set = true;
    }
    const size_t smem = ((size_t(5 * cnt + 4) * 4 + 15) & ~size_t(15)) + size_t(2 * cnt) * kSwpCols * sizeof(T2);
    dim3 grid(ceil_div(ncols, kSwpCols), F);
    ProfScope ps(PK_LASWP, 0.0, st);
    laswp_kernel<T2><<<grid, kSwpThreads, smem, st>>>(G, sG, ld, j, cnt, ipiv, sP, a0, a1, b0, b1);
}

template <typename R>
void launch_trsm(typename Cplx<R>::T* G, int64_t sG, int ld, int F, int j, int cnt, int c0, int c1,
                 cudaStream_t st) {
    using T2 = typename Cplx<R>::T;
    if (c1 <= c0 || cnt <= 1) return;
    const size_t smem = size_t(cnt) * cnt * sizeof(T2) + size_t(cnt) * kTrsmThreads * sizeof(T2);
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(trsm_kernel<T2>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        attr_set = true;
    }
    dim3 grid(ceil_div(c1 - c0, kTrsmThreads), F);
    ProfScope ps(PK_TRSM, 8.0 * F * double(cnt) * cnt / 2.0 * (c1 - c0), st);
    if (cnt == 16) {
        trsm_reg_kernel<T2, 16><<<grid, kTrsmThreads, 0, st>>>(G, sG, ld, j, c0, c1);
        return;
    }
    if constexpr (sizeof(R) == 4) {
        if (cnt == 32) {
            trsm_reg_kernel<T2, 32><<<grid, kTrsmThreads, 0, st>>>(G, sG, ld, j, c0, c1);
            return;
        }
    }
    trsm_kernel<T2><<<grid, kTrsmThreads, smem, st>>>(G, sG, ld, j, cnt, c0, c1);
}

template <typename R>
void launch_gemm_update(typename Cplx<R>::T* G, int64_t sG, int ld, int F, int r0, int r1, int c0, int c1, int k0,
                        int K, cudaStream_t st) {
    using T2 = typename Cplx<R>::T;
    if (r1 <= r0 || c1 <= c0 || K <= 0) return;
    if constexpr (sizeof(R) == 4) {
        launch_cgemm_f32(G, sG, ld, F, r0, r1, c0, c1, k0, K, st);
        return;
    }
    dim3 grid(ceil_div(c1 - c0, kBN), ceil_div(r1 - r0, kBM), F);
    ProfScope ps(PK_GEMM, 8.0 * F * double(r1 - r0) * double(c1 - c0) * K, st);
    gemm_update_kernel<T2><<<grid, kGemmThreads, 0, st>>>(G, sG, ld, r0, r1, c0, c1, k0, K);
}

template <typename R>
void trailing_update(typename Cplx<R>::T* G, int64_t sG, int ld, int F, int r0, int r1, int c0, int c1, int k0, int K,
                     const TcCtx* tc, cudaStream_t st) {
    if constexpr (sizeof(R) == 4) {
        // narrow updates (fewer than 64 complex columns) would waste most of a 128-wide tensor tile
        if (tc && c1 - c0 >= kTcMinCols && launch_tc_update(G, sG, ld, F, r0, r1, c0, c1, k0, K, *tc, st)) return;
    }
    launch_gemm_update<R>(G, sG, ld, F, r0, r1, c0, c1, k0, K, st);
}

// rows per block of the left-looking solve U12 = L11^-1 A12 of the columns right of the pivots
constexpr int kLazyTrsmRows = 128;

// smallest batch whose outer panels are factored recursively (factor_outer_cols).  The recursion
// moves less of C but solves triangles of up to 64 rows where the flat loop solves 16-row ones;
// those are latency-bound, so a few matrices are faster with the flat loop (measured on config-2
// windows: batch 96 22.7 vs 23.0 ms, batch 1 5.2 vs 4.9 ms).
constexpr int kRecursiveMinBatch = 32;

// Columns [j, j + w) of the outer panel [J, J + nb), factored recursively: the left half (a
// multiple of the panel width) is factored, its U rows are solved for the right half's columns
// (32-row triangles joined by updates), the right half takes the update with K = the left
// half's width, and is factored in turn.  The leaves are panels of at most nbw columns, whose
// interchanges reach the whole outer panel.  The arithmetic is that of the right-looking order
// over nbw-column panels; the updates of C inside the outer panel shrink from
// (nb - nbw) + (nb - 2 nbw) + ... columns of C read and written to nb / 2 per level.
template <typename R>
void factor_outer_cols(typename Cplx<R>::T* G, int64_t sG, int ld, int F, int m, int J, int nb, int j, int w,
                       int nbw, int32_t* ipiv, int64_t sP, int32_t* status, const TcCtx* tc, cudaStream_t st) {
    if (w <= nbw) {
        launch_panel<R>(G, sG, ld, F, m, j, w, ipiv, sP, status, J, J + nb, st);
        return;
    }
    const int h = (w / 2 + nbw - 1) / nbw * nbw;
    factor_outer_cols<R>(G, sG, ld, F, m, J, nb, j, h, nbw, ipiv, sP, status, tc, st);
    for (int r = 0; r < h; r += kTrsmMaxRows) {
        const int cnt = std::min(kTrsmMaxRows, h - r);
        launch_trsm<R>(G, sG, ld, F, j + r, cnt, j + h, j + w, st);
        if (r + cnt < h) launch_gemm_update<R>(G, sG, ld, F, j + r + cnt, j + h, j + h, j + w, j + r, cnt, st);
    }
    trailing_update<R>(G, sG, ld, F, j + h, m, j + h, j + w, j, h, tc, st);
    factor_outer_cols<R>(G, sG, ld, F, m, J, nb, j + h, w - h, nbw, ipiv, sP, status, tc, st);
}

// Partial LU of the first npiv columns, right-looking in outer panels of NB columns, with the
// updates of the outer panels restricted to the pivot columns [0, npiv).  The columns right of
// them, [npiv, ncols), only receive their row interchanges while the pivot columns are
// factored; afterwards U12 = L11^-1 A12 is solved left-looking in 128-row blocks (each block
// first takes the product of the multipliers and all rows above it, K up to npiv) and the
// Schur complement A22 -= L21 U12 is one update with K = npiv.  The arithmetic is that of the
// right-looking order (the same pivots; sums in a different order), but most of it runs in
// updates with a long K.  With tensor cores the outer-panel updates (K = 128) and every update of
// the lazy phase run there; the rows of U12 are packed for them once, 32 rows at a time as they
// are solved, and every later update reads them from there.  Inside an outer panel the columns
// are factored recursively for batches of kRecursiveMinBatch or more (factor_outer_cols; its
// updates of at least 64 columns go to the tensor cores as well, the narrower ones stay on the
// FP32 pipe), right-looking over nbw-column panels for smaller batches.
template <typename R>
void partial_lu(typename Cplx<R>::T* G, int64_t sG, int ld, int F, int m, int ncols, int npiv, int32_t* ipiv,
                int64_t sP, int32_t* status, cudaStream_t st, const TcCtx* tc) {
    const int NB = outer_nb<R>();
    const int nbw = std::min(panel_width<R>(m), NB);
    for (int J = 0; J < npiv; J += NB) {
        const int nb = std::min(NB, npiv - J);
        if (F >= kRecursiveMinBatch) {
            factor_outer_cols<R>(G, sG, ld, F, m, J, nb, J, nb, nbw, ipiv, sP, status, tc, st);
        } else {
            for (int j = J; j < J + nb; j += nbw) {   // right-looking over nbw-column panels
                const int w = std::min(nbw, J + nb - j);
                launch_panel<R>(G, sG, ld, F, m, j, w, ipiv, sP, status, J, J + nb, st);
                if (j + w < J + nb) {
                    launch_trsm<R>(G, sG, ld, F, j, w, j + w, J + nb, st);
                    launch_gemm_update<R>(G, sG, ld, F, j + w, m, j + w, J + nb, j, w, st);
                }
            }
        }
        launch_laswp<R>(G, sG, ld, F, J, nb, ipiv, sP, 0, J, J + nb, ncols, st);
        if (J + nb < npiv) {
            for (int r = 0; r < nb; r += kTrsmMaxRows) {   // the outer panel's U rows, 32-row triangles
                const int cnt = std::min(kTrsmMaxRows, nb - r);
                launch_trsm<R>(G, sG, ld, F, J + r, cnt, J + nb, npiv, st);
                if (r + cnt < nb)
                    launch_gemm_update<R>(G, sG, ld, F, J + r + cnt, J + nb, J + nb, npiv, J + r, cnt, st);
            }
            trailing_update<R>(G, sG, ld, F, J + nb, m, J + nb, npiv, J, nb, tc, st);
        }
    }
    if (npiv < ncols) {
        TcCtx lz;
        bool lazy = false;
        if constexpr (sizeof(R) == 4) {
            if (tc) {
                lz = *tc;
                lazy = tc_begin_lazy(G, sG, ld, F, npiv, npiv, ncols, lz, st);
            }
        }
        // C[r0:r1, npiv:ncols] -= G[r0:r1, k0:k0+K] U12[k0:k0+K, :]
        auto update = [&](int r0, int r1, int k0, int K) {
            if constexpr (sizeof(R) == 4) {
                if (lazy && launch_tc_update_lazy(G, sG, ld, F, r0, r1, k0, K, lz, st)) return;
                lazy = false;   // the packed rows are not kept up to date from here on
            }
            trailing_update<R>(G, sG, ld, F, r0, r1, npiv, ncols, k0, K, tc, st);
        };
        for (int I = 0; I < npiv; I += kLazyTrsmRows) {
            const int tb = std::min(kLazyTrsmRows, npiv - I);
            if (I > 0) update(I, I + tb, 0, I);
            for (int r = 0; r < tb; r += kTrsmMaxRows) {   // 32-row triangles joined by updates
                const int cnt = std::min(kTrsmMaxRows, tb - r);
                launch_trsm<R>(G, sG, ld, F, I + r, cnt, npiv, ncols, st);
                if constexpr (sizeof(R) == 4) {
                    if (lazy) tc_pack_b_rows(G, sG, ld, F, I + r, I + r + cnt, lz, st);
                }
                if (r + cnt < tb) update(I + r + cnt, I + tb, I + r, cnt);
            }
        }
        if (npiv < m) update(npiv, m, 0, npiv);
    }
}

template <typename R>
void launch_slab_shift(typename Cplx<R>::T* G, int64_t sG, int F, int b, int m, typename Cplx<R>::T* U, int64_t sU,
                       typename Cplx<R>::T* L, int64_t sL, const int32_t* ipiv, int64_t sP, int32_t* perm,
                       int64_t sPerm, cudaStream_t st) {
    using T2 = typename Cplx<R>::T;
    dim3 grid(ceil_div(int64_t(b) * 3 * b, 256), F);
    ProfScope ps(PK_SHIFT, 0.0, st);
    slab_shift_kernel<T2><<<grid, 256, 0, st>>>(G, sG, b, m, U, sU, L, sL);
    ProfScope ps2(PK_SHIFT, 0.0, st);
    perm_kernel<<<F, 256, size_t(m) * sizeof(int32_t), st>>>(ipiv, sP, perm, sPerm, b, m);
}

template <typename R>
void launch_backsub(typename Cplx<R>::T* G, int64_t sG, int ld, int F, int n, int c0, int nrhs, cudaStream_t st) {
    using T2 = typename Cplx<R>::T;
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(backsub_kernel<T2>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
        attr_set = true;
    }
    for (int cc = 0; cc < nrhs; cc += kRmax) {
        const int nc = std::min(kRmax, nrhs - cc);
        ProfScope ps(PK_SOLVE, 8.0 * F * nc * double(n) * n / 2.0, st);
        backsub_kernel<T2><<<F, kSolveThreads, size_t(n) * nc * sizeof(T2), st>>>(G, sG, ld, n, c0 + cc, nc);
    }
}

#define FSI_INSTANTIATE(R)                                                                                           \
    template void launch_form_rows<R>(const DevModel&, Cplx<R>::T*, int64_t, int, int, const double*, int, int, int, \
                                      int, cudaStream_t);                                                            \
    template int panel_width<R>(int);                                                                                \
    template void launch_panel<R>(Cplx<R>::T*, int64_t, int, int, int, int, int, int32_t*, int64_t, int32_t*, int, \
                                  int, cudaStream_t);                                                                \
    template void launch_laswp<R>(Cplx<R>::T*, int64_t, int, int, int, int, const int32_t*, int64_t, int, int, int, \
                                  int, cudaStream_t);                                                                \
    template void launch_trsm<R>(Cplx<R>::T*, int64_t, int, int, int, int, int, int, cudaStream_t);                 \
    template void launch_gemm_update<R>(Cplx<R>::T*, int64_t, int, int, int, int, int, int, int, int, cudaStream_t); \
    template void partial_lu<R>(Cplx<R>::T*, int64_t, int, int, int, int, int, int32_t*, int64_t, int32_t*,         \
                                cudaStream_t, const TcCtx*);                                                         \
    template void launch_slab_shift<R>(Cplx<R>::T*, int64_t, int, int, int, Cplx<R>::T*, int64_t, Cplx<R>::T*,      \
                                       int64_t, const int32_t*, int64_t, int32_t*, int64_t, cudaStream_t);           \
    template void launch_backsub<R>(Cplx<R>::T*, int64_t, int, int, int, int, int, cudaStream_t);

FSI_INSTANTIATE(float)
FSI_INSTANTIATE(double)

}  // namespace fsi
