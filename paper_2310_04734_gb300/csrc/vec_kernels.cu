// FP64 vector kernels of the iterative refinement: the sparse residual
// r = f - A(w) x with A(w) = K + i w D - w^2 M formed entry by entry from the
// CSR values (paper Sec. 3.3, Eq. 8), conversions between the FP64 iterate and
// the low-precision correction, and the receiver read-out with SPL.
#include <cmath>

#include "kernels.cuh"
#include "prof.h"

namespace fsi {

namespace {

constexpr int kResRmax = 8;

__global__ void residual_kernel(DevModel m, const double* omega, double omega0, const double2* x, int64_t sX,
                                const double2* Fm, int nrhs, double2* r, int64_t sR, double* norms, int nstride,
                                int ncol0, bool scaled, double* absn) {
    const int f = blockIdx.y;
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const double w = omega ? omega[f] : omega0;
    double2 acc[kResRmax];
#pragma unroll
    for (int c = 0; c < kResRmax; ++c) acc[c] = make_double2(0.0, 0.0);
    double nrm[kResRmax], sab[kResRmax], anr[kResRmax];
#pragma unroll
    for (int c = 0; c < kResRmax; ++c) nrm[c] = sab[c] = anr[c] = 0.0;
    if (i < m.n) {
        if (x) {
            const double2* xf = x + f * sX;
            const int e1 = m.rowptr[i + 1];
            for (int e = m.rowptr[i]; e < e1; ++e) {
                const int64_t col = m.col[e];
                double2 a = a_entry(m, e, w);
                if (scaled) {
                    const double s = col_scale(m, col, w);
                    a.x *= s;
                    a.y *= s;
                }
#pragma unroll
                for (int c = 0; c < kResRmax; ++c)
                    if (c < nrhs) cfma(acc[c], a, xf[c * m.n + col]);
                if (absn) {
                    const double aa = hypot(a.x, a.y);
#pragma unroll
                    for (int c = 0; c < kResRmax; ++c)
                        if (c < nrhs) {
                            const double2 xv = xf[c * m.n + col];
                            sab[c] += aa * hypot(xv.x, xv.y);
                        }
                }
            }
        }
        const double rs = scaled ? row_scale(m, i, w) : 1.0;
        double2* rf = r + f * sR;
#pragma unroll
        for (int c = 0; c < kResRmax; ++c) {
            if (c >= nrhs) break;
            const double2 fv = Fm[c * m.n + i];
            const double2 v = make_double2(rs * (fv.x - acc[c].x), rs * (fv.y - acc[c].y));
            rf[c * m.n + i] = v;
            nrm[c] = v.x * v.x + v.y * v.y;
            const double t = rs * (sab[c] + hypot(fv.x, fv.y));
            anr[c] = t * t;
        }
    }
    if (absn) {
        const int lane = threadIdx.x & 31;
#pragma unroll
        for (int c = 0; c < kResRmax; ++c) {
            if (c >= nrhs) break;
            double v = anr[c];
            for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
            if (lane == 0 && v != 0.0) atomicAdd(&absn[f * nstride + ncol0 + c], v);
        }
    }
    if (norms) {
        const int lane = threadIdx.x & 31;
#pragma unroll
        for (int c = 0; c < kResRmax; ++c) {
            if (c >= nrhs) break;
            double v = nrm[c];
            for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
            if (lane == 0 && v != 0.0) atomicAdd(&norms[f * nstride + ncol0 + c], v);
        }
    }
}

template <typename T2>
__global__ void to_low_kernel(const double2* r, int64_t sR, const double* norms, T2* y, int64_t sY, int64_t n,
                              int nrhs) {
    using R = decltype(T2::x);
    const int f = blockIdx.y;
    const int64_t q = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (q >= n * nrhs) return;
    const int c = int(q / n);
    const double s = sqrt(norms[f * nrhs + c]);
    const double inv = s > 0.0 ? 1.0 / s : 0.0;
    const double2 v = r[f * sR + q];
    y[f * sY + q] = mk<T2>(R(v.x * inv), R(v.y * inv));
}

template <typename T2>
__global__ void update_kernel(double2* x, int64_t sX, const double* norms, const T2* y, int64_t sY, int64_t n,
                              int nrhs, const int32_t* active) {
    const int f = blockIdx.y;
    const int64_t q = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (q >= n * nrhs) return;
    const int c = int(q / n);
    if (active && !active[f * nrhs + c]) return;
    const double s = sqrt(norms[f * nrhs + c]);
    const T2 d = y[f * sY + q];
    double2& xv = x[f * sX + q];
    xv.x += s * double(d.x);
    xv.y += s * double(d.y);
}

__global__ void receivers_kernel(DevModel m, const double* omega, const double2* x, int64_t sX, const int32_t* rcv,
                                 int nrcv, int nrhs, double2* p, double* spl) {
    const int f = blockIdx.y;
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nrcv * nrhs) return;
    const int ir = q / nrhs, c = q - ir * nrhs;
    const int64_t g = rcv[ir];
    const double w = omega[f];
    const double cs = col_scale(m, g, w);
    const double2 v = x[f * sX + c * m.n + g];
    const double2 pv = make_double2(cs * v.x, cs * v.y);
    const int64_t o = (int64_t(f) * nrcv + ir) * nrhs + c;
    p[o] = pv;
    if (spl) spl[o] = 20.0 * log10(sqrt(pv.x * pv.x + pv.y * pv.y) / (sqrt(2.0) * 2e-5));
}

inline unsigned ceil_div(int64_t a, int64_t b) { return unsigned((a + b - 1) / b); }

}  // namespace

void launch_residual(const DevModel& m, const double* d_omega, double omega0, int F, const double2* x, int64_t sX,
                     const double2* Fm, int nrhs, double2* r, int64_t sR, double* norms, bool scaled,
                     cudaStream_t st, double* absn) {
    for (int c0 = 0; c0 < nrhs; c0 += kResRmax) {
        const int nc = nrhs - c0 < kResRmax ? nrhs - c0 : kResRmax;
        dim3 grid(ceil_div(m.n, 256), F);
        ProfScope ps(PK_RESID, 0.0, st);
        residual_kernel<<<grid, 256, 0, st>>>(m, d_omega, omega0, x ? x + c0 * m.n : nullptr, sX, Fm + c0 * m.n, nc,
                                              r + c0 * m.n, sR, norms, nrhs, c0, scaled, absn);
    }
}

template <typename R>
void launch_to_low(const double2* r, int64_t sR, const double* norms, typename Cplx<R>::T* y, int64_t sY, int64_t n,
                   int nrhs, int F, cudaStream_t st) {
    dim3 grid(ceil_div(n * nrhs, 256), F);
    ProfScope ps(PK_RESID, 0.0, st);
    to_low_kernel<<<grid, 256, 0, st>>>(r, sR, norms, y, sY, n, nrhs);
}

template <typename R>
void launch_update(double2* x, int64_t sX, const double* norms, const typename Cplx<R>::T* y, int64_t sY, int64_t n,
                   int nrhs, int F, const int32_t* active, cudaStream_t st) {
    dim3 grid(ceil_div(n * nrhs, 256), F);
    ProfScope ps(PK_RESID, 0.0, st);
    update_kernel<<<grid, 256, 0, st>>>(x, sX, norms, y, sY, n, nrhs, active);
}

void launch_receivers(const DevModel& m, const double* d_omega, int F, const double2* x, int64_t sX,
                      const int32_t* rcv, int nrcv, int nrhs, double2* p, double* spl, cudaStream_t st) {
    dim3 grid(ceil_div(int64_t(nrcv) * nrhs, 128), F);
    ProfScope ps(PK_RESID, 0.0, st);
    receivers_kernel<<<grid, 128, 0, st>>>(m, d_omega, x, sX, rcv, nrcv, nrhs, p, spl);
}

template void launch_to_low<float>(const double2*, int64_t, const double*, float2*, int64_t, int64_t, int, int,
                                   cudaStream_t);
template void launch_to_low<double>(const double2*, int64_t, const double*, double2*, int64_t, int64_t, int, int,
                                    cudaStream_t);
template void launch_update<float>(double2*, int64_t, const double*, const float2*, int64_t, int64_t, int, int,
                                   const int32_t*, cudaStream_t);
template void launch_update<double>(double2*, int64_t, const double*, const double2*, int64_t, int64_t, int, int,
                                    const int32_t*, cudaStream_t);

}  // namespace fsi
