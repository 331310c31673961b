// Reduced sweeps of many reduced models of uneven size in one persistent launch
// (the online phase of the paper's ROM, Sec. 3.3 / Eq. 11, for a batch of design
// variants).
//
// Work items are (model, frequency) pairs numbered model by model; CTAs take
// items from a global counter until none is left, so models of different k
// share the launch without a per-model grid.  Each item:
//   A = K_R + i w D_R - w^2 M_R (FP64 inputs), equilibrated by row then column
//   maxima, factored by LU with partial pivoting in FP32 in shared memory;
//   x from the factor, then refinement steps x += C LU^-1 (R (f_R - A x)) with
//   the residual in FP64 from the FP64 reduced matrices, until the correction is
//   at FP64 rounding level (at most 8); p = C_R x, SPL.
// The launch only enqueues a memset of the counter and the kernel (no host
// synchronisation, no allocation), so it can be captured into a CUDA graph.
// A status word per item records a zero or non-finite pivot, or a refinement that
// did not converge (a reduced system too ill-conditioned for its FP32 factor; the
// caller re-solves those items in FP64).
#include <cuda_runtime.h>

#include <algorithm>
#include <string>

#include "fsi_internal.h"

namespace fsi {

namespace {

constexpr int kMT = 256;          // threads per CTA
constexpr int kKMax = 128;        // largest reduced order
constexpr int kRMax = 4;          // load columns per model
constexpr int kRefine = 8;        // FP64 refinement steps at most (stop when the correction is at rounding level)

struct MultiSmem {
    float2 A[kKMax * kKMax];      // row-major, equilibrated, then L\U
    double2 x[kKMax * kRMax];     // solution (FP64), [j][c]
    double2 r[kKMax * kRMax];     // residual / correction
    float2 y[kKMax * kRMax];      // FP32 right-hand side of a solve
    double rs[kKMax], cs[kKMax];  // row / column scales
    int piv[kKMax];
    float rv[kMT / 32];
    int ri[kMT / 32];
    int item;
    int bad;
};

__device__ __forceinline__ double2 cmulD(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// A_e = K + i w D - w^2 M (column-major k x k inputs, entry (i, j) at j*k + i)
__device__ __forceinline__ double2 a_red(const fsi_rom_item& it, int i, int j, double w) {
    const int64_t e = int64_t(j) * it.k + i;
    const double2 kk = reinterpret_cast<const double2*>(it.KR)[e];
    const double2 dd = reinterpret_cast<const double2*>(it.DR)[e];
    const double2 mm = reinterpret_cast<const double2*>(it.MR)[e];
    return make_double2(kk.x - w * dd.y - w * w * mm.x, kk.y + w * dd.x - w * w * mm.y);
}

// in-place y <- U^-1 L^-1 P y for the factor in S.A (nr columns), FP32
__device__ void lu_solve(MultiSmem& S, int k, int nr) {
    const int tid = threadIdx.x;
    // row interchanges in pivot order (one thread per column)
    if (tid < nr)
        for (int j = 0; j < k; ++j) {
            const int p = S.piv[j];
            if (p != j) {
                const float2 t = S.y[j * kRMax + tid];
                S.y[j * kRMax + tid] = S.y[p * kRMax + tid];
                S.y[p * kRMax + tid] = t;
            }
        }
    __syncthreads();
    // forward (unit lower): column-oriented, rows below j updated in parallel
    for (int j = 0; j < k; ++j) {
        for (int q = tid; q < (k - j - 1) * nr; q += blockDim.x) {
            const int i = j + 1 + q / nr, c = q - (q / nr) * nr;
            const float2 l = S.A[i * kKMax + j], v = S.y[j * kRMax + c];
            float2& t = S.y[i * kRMax + c];
            t.x -= l.x * v.x - l.y * v.y;
            t.y -= l.x * v.y + l.y * v.x;
        }
        __syncthreads();
    }
    // backward
    for (int j = k - 1; j >= 0; --j) {
        if (tid < nr) {
            const float2 d = S.A[j * kKMax + j];
            const float den = d.x * d.x + d.y * d.y;
            const float2 v = S.y[j * kRMax + tid];
            S.y[j * kRMax + tid] = make_float2((v.x * d.x + v.y * d.y) / den, (v.y * d.x - v.x * d.y) / den);
        }
        __syncthreads();
        for (int q = tid; q < j * nr; q += blockDim.x) {
            const int i = q / nr, c = q - i * nr;
            const float2 u = S.A[i * kKMax + j], v = S.y[j * kRMax + c];
            float2& t = S.y[i * kRMax + c];
            t.x -= u.x * v.x - u.y * v.y;
            t.y -= u.x * v.y + u.y * v.x;
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kMT) rom_multi_kernel(const fsi_rom_item* items, int nvar, const int32_t* off,
                                                        int total, int* counter, int32_t* status) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    MultiSmem& S = *reinterpret_cast<MultiSmem*>(smem_raw);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (;;) {
        if (tid == 0) S.item = atomicAdd(counter, 1);
        __syncthreads();
        const int g = S.item;
        if (g >= total) return;
        // model of item g: off is the prefix sum of the models' frequency counts
        int lo = 0, hi = nvar - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (off[mid] <= g) lo = mid;
            else hi = mid - 1;
        }
        const fsi_rom_item it = items[lo];
        const int fi = g - off[lo];
        const int k = it.k, nr = it.nrhs;
        if (k <= 0 || k > kKMax || nr <= 0 || nr > kRMax || it.nrcv <= 0) {   // descriptor out of range
            if (tid == 0 && status) status[g] = 2;
            __syncthreads();
            continue;
        }
        const double w = 2.0 * M_PI * it.f_hz[fi];
        if (tid == 0) S.bad = 0;
        // equilibration scales: rows, then columns of the row-scaled matrix
        for (int i = tid; i < k; i += blockDim.x) {
            double mx = 0.0;
            for (int j = 0; j < k; ++j) {
                const double2 a = a_red(it, i, j, w);
                mx = fmax(mx, hypot(a.x, a.y));
            }
            S.rs[i] = mx > 0.0 ? 1.0 / mx : 1.0;
        }
        __syncthreads();
        for (int j = tid; j < k; j += blockDim.x) {
            double mx = 0.0;
            for (int i = 0; i < k; ++i) {
                const double2 a = a_red(it, i, j, w);
                mx = fmax(mx, S.rs[i] * hypot(a.x, a.y));
            }
            S.cs[j] = mx > 0.0 ? 1.0 / mx : 1.0;
        }
        __syncthreads();
        for (int q = tid; q < k * k; q += blockDim.x) {
            const int i = q / k, j = q - i * k;
            const double2 a = a_red(it, i, j, w);
            const double s = S.rs[i] * S.cs[j];
            S.A[i * kKMax + j] = make_float2(float(s * a.x), float(s * a.y));
        }
        __syncthreads();
        // LU with partial pivoting
        for (int j = 0; j < k; ++j) {
            float best = -1.f;
            int bi = j;
            for (int i = j + tid; i < k; i += blockDim.x) {
                const float2 a = S.A[i * kKMax + j];
                const float m = a.x * a.x + a.y * a.y;
                if (m > best) {
                    best = m;
                    bi = i;
                }
            }
            for (int o = 16; o > 0; o >>= 1) {
                const float ob = __shfl_down_sync(0xffffffffu, best, o);
                const int oi = __shfl_down_sync(0xffffffffu, bi, o);
                if (ob > best || (ob == best && oi < bi)) {
                    best = ob;
                    bi = oi;
                }
            }
            if (lane == 0) {
                S.rv[warp] = best;
                S.ri[warp] = bi;
            }
            __syncthreads();
            if (tid == 0) {
                float b = S.rv[0];
                int p = S.ri[0];
                for (int q = 1; q < int(blockDim.x >> 5); ++q)
                    if (S.rv[q] > b || (S.rv[q] == b && S.ri[q] < p)) {
                        b = S.rv[q];
                        p = S.ri[q];
                    }
                if (!(b > 0.f) || !isfinite(b)) {
                    S.bad = 1;
                    p = j;
                }
                S.piv[j] = p;
            }
            __syncthreads();
            const int p = S.piv[j];
            if (p != j)
                for (int c = tid; c < k; c += blockDim.x) {
                    const float2 t = S.A[j * kKMax + c];
                    S.A[j * kKMax + c] = S.A[p * kKMax + c];
                    S.A[p * kKMax + c] = t;
                }
            __syncthreads();
            const float2 d = S.A[j * kKMax + j];
            const float den = d.x * d.x + d.y * d.y;
            if (den > 0.f) {
                for (int i = j + 1 + tid; i < k; i += blockDim.x) {
                    const float2 a = S.A[i * kKMax + j];
                    S.A[i * kKMax + j] = make_float2((a.x * d.x + a.y * d.y) / den, (a.y * d.x - a.x * d.y) / den);
                }
            }
            __syncthreads();
            const int rows = k - j - 1;
            for (int q = tid; q < rows * rows; q += blockDim.x) {
                const int i = j + 1 + q / rows, c = j + 1 + (q - (q / rows) * rows);
                const float2 l = S.A[i * kKMax + j], u = S.A[j * kKMax + c];
                float2& t = S.A[i * kKMax + c];
                t.x -= l.x * u.x - l.y * u.y;
                t.y -= l.x * u.y + l.y * u.x;
            }
            __syncthreads();
        }
        // x = 0; r = f_R; then refinement passes: y = R r, solve, x += C y, r = f_R - A x (FP64)
        const double2* fR = reinterpret_cast<const double2*>(it.fR);
        for (int q = tid; q < k * nr; q += blockDim.x) {
            const int i = q / nr, c = q - i * nr;
            S.x[i * kRMax + c] = make_double2(0.0, 0.0);
            S.r[i * kRMax + c] = fR[int64_t(c) * k + i];
        }
        __syncthreads();
        bool conv = false;
        for (int pass = 0; pass <= kRefine; ++pass) {
            for (int q = tid; q < k * nr; q += blockDim.x) {
                const int i = q / nr, c = q - i * nr;
                const double2 v = S.r[i * kRMax + c];
                S.y[i * kRMax + c] = make_float2(float(S.rs[i] * v.x), float(S.rs[i] * v.y));
            }
            __syncthreads();
            lu_solve(S, k, nr);
            float dmax = 0.f, xmax = 0.f;
            for (int q = tid; q < k * nr; q += blockDim.x) {
                const int i = q / nr, c = q - i * nr;
                const float2 v = S.y[i * kRMax + c];
                double2& xv = S.x[i * kRMax + c];
                const double dx = S.cs[i] * double(v.x), dy = S.cs[i] * double(v.y);
                xv.x += dx;
                xv.y += dy;
                dmax = fmaxf(dmax, float(fabs(dx) + fabs(dy)));
                xmax = fmaxf(xmax, float(fabs(xv.x) + fabs(xv.y)));
            }
            for (int o = 16; o > 0; o >>= 1) {
                dmax = fmaxf(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
                xmax = fmaxf(xmax, __shfl_xor_sync(0xffffffffu, xmax, o));
            }
            if (lane == 0) {
                S.rv[warp] = dmax;
                S.ri[warp] = __float_as_int(xmax);
            }
            __syncthreads();
            float dall = 0.f, xall = 0.f;
            for (int q = 0; q < int(blockDim.x >> 5); ++q) {
                dall = fmaxf(dall, S.rv[q]);
                xall = fmaxf(xall, __int_as_float(S.ri[q]));
            }
            __syncthreads();
            conv = dall <= 1e-12f * xall;
            if (pass == kRefine || dall <= 1e-15f * xall) break;
            for (int q = tid; q < k * nr; q += blockDim.x) {
                const int i = q / nr, c = q - i * nr;
                double2 acc = fR[int64_t(c) * k + i];
                for (int j = 0; j < k; ++j) {
                    const double2 t = cmulD(a_red(it, i, j, w), S.x[j * kRMax + c]);
                    acc.x -= t.x;
                    acc.y -= t.y;
                }
                S.r[i * kRMax + c] = acc;
            }
            __syncthreads();
        }
        // receivers
        const double2* CR = reinterpret_cast<const double2*>(it.CR);
        double2* p = reinterpret_cast<double2*>(it.p_out) + int64_t(fi) * it.nrcv * nr;
        for (int q = tid; q < it.nrcv * nr; q += blockDim.x) {
            const int ir = q / nr, c = q - ir * nr;
            double2 acc = make_double2(0.0, 0.0);
            for (int j = 0; j < k; ++j) {
                const double2 t = cmulD(CR[int64_t(j) * it.nrcv + ir], S.x[j * kRMax + c]);
                acc.x += t.x;
                acc.y += t.y;
            }
            p[q] = acc;
            if (it.spl_out)
                it.spl_out[int64_t(fi) * it.nrcv * nr + q] =
                    20.0 * log10(sqrt(acc.x * acc.x + acc.y * acc.y) / (sqrt(2.0) * 2e-5));
        }
        if (tid == 0 && status) status[g] = S.bad ? 1 : (conv ? 0 : 3);
        __syncthreads();
    }
}

}  // namespace

}  // namespace fsi

using namespace fsi;

extern "C" {

fsi_status rom_multi_sweep(const fsi_rom_item* items, int nvar, const int32_t* offsets, int total, int* counter,
                           int32_t* status, void* stream) {
    if (!(items && offsets && counter && nvar > 0 && total > 0)) {
        set_error("rom_multi_sweep: bad arguments");
        return FSI_EINVAL;
    }
    static bool attr = false;
    static int grid = 0;
    if (!attr) {
        cudaFuncSetAttribute(rom_multi_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sizeof(MultiSmem)));
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        grid = sms > 0 ? sms : 1;
        attr = true;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(int), st);
    if (e == cudaSuccess) {
        rom_multi_kernel<<<std::min(grid, total), kMT, sizeof(MultiSmem), st>>>(items, nvar, offsets, total, counter,
                                                                              status);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        set_error(std::string("rom_multi_sweep: ") + cudaGetErrorString(e));
        return FSI_ECUDA;
    }
    return FSI_OK;
}

}  // extern "C"
