// FP64 vector kernels of the iterative refinement: the sparse residual
// r = f - A(w) x with A(w) = K + i w D - w^2 M formed entry by entry from the
// CSR values (paper Sec. 3.3, Eq. 8), conversions between the FP64 iterate and
// the low-precision correction, and the receiver read-out with SPL.
#include <cmath>

#include "csr_rows.cuh"
#include "kernels.cuh"
#include "prof.h"

namespace fsi {

namespace {


// r_c = rs o (f_c - A(w) (cs o x_c)) (scaled) or f_c - A(w) x_c for the R load columns of
// this launch (R a power of two), frequency f = blockIdx.y; norms[f][ncol0 + c] += |r_c|^2
// and, with absn, absn[f][ncol0 + c] += |rs o (|A| |cs o x_c| + |f_c|)|^2 (the rounding
// level of the residual).  Row groups of kRowLanes lanes; after the reduce-scatter each
// lane owns kept_slots<R> load columns of its row.
template <int R, bool scaled>
__global__ void __launch_bounds__(kRowThreads) residual_kernel(DevModel m, const double* omega, double omega0,
                                                               const double2* x, int64_t sX, const double2* Fm,
                                                               int64_t sF, double2* r, int64_t sR, double* norms,
                                                               int nstride, int ncol0, double* absn) {
    constexpr int KS = kept_slots<R>();
    const int f = blockIdx.y;
    const double w = omega ? omega[f] : omega0, w2 = w * w, inv_w = 1.0 / w;
    const int g = threadIdx.x & (kRowLanes - 1);
    const int c0 = slot_base<R>(g);
    const bool writer = slot_writer<R>(g);
    const double2* xf = x ? x + f * sX : nullptr;
    const double2* Ff = Fm + f * sF;   // sF = 0: one right-hand side for every frequency
    double2* rf = r + f * sR;
    double nrm[KS], anr[KS];
#pragma unroll
    for (int q = 0; q < KS; ++q) nrm[q] = anr[q] = 0.0;
    for (int64_t base = int64_t(blockIdx.x) * kRowsPerCta; base < m.n; base += int64_t(gridDim.x) * kRowsPerCta) {
        const int64_t i = base + threadIdx.x / kRowLanes;
        const bool valid = i < m.n;
        double2 acc[R];
        double sab[R];
#pragma unroll
        for (int c = 0; c < R; ++c) {
            acc[c] = make_double2(0.0, 0.0);
            sab[c] = 0.0;
        }
        if (valid && xf) {
            const int e1 = __ldg(m.rowptr + i + 1);
            for (int e = __ldg(m.rowptr + i) + g; e < e1; e += kRowLanes) {
                const int64_t col = __ldg(m.col + e);
                double2 a = a_entry_ld(m, e, w, w2);
                if (scaled) {
                    const double s = col_scale(m, col, w);
                    a.x *= s;
                    a.y *= s;
                }
#pragma unroll
                for (int c = 0; c < R; ++c) cfma(acc[c], a, xf[c * m.n + col]);
                if (absn) {
                    const double aa = hypot(a.x, a.y);
#pragma unroll
                    for (int c = 0; c < R; ++c) {
                        const double2 xv = xf[c * m.n + col];
                        sab[c] = fma(aa, hypot(xv.x, xv.y), sab[c]);
                    }
                }
            }
        }
        group_reduce_scatter<R>(acc, g);
        if (absn) group_reduce_scatter<R>(sab, g);
        if (valid && writer) {
            const double rs = scaled ? row_scale_inv(m, i, inv_w) : 1.0;
#pragma unroll
            for (int q = 0; q < KS; ++q) {
                const int c = c0 + q;
                const double2 fv = Ff[c * m.n + i];
                const double2 v = make_double2(rs * (fv.x - acc[q].x), rs * (fv.y - acc[q].y));
                rf[c * m.n + i] = v;
                nrm[q] = fma(v.x, v.x, fma(v.y, v.y, nrm[q]));
                if (absn) {
                    const double t = rs * (sab[q] + hypot(fv.x, fv.y));
                    anr[q] = fma(t, t, anr[q]);
                }
            }
        }
    }
    // per load column: shared-memory sums over the CTA, then one global atomic per column
    __shared__ double red[2][R];
    if (threadIdx.x < 2 * R) (&red[0][0])[threadIdx.x] = 0.0;
    __syncthreads();
    if (writer) {
#pragma unroll
        for (int q = 0; q < KS; ++q) {
            if (nrm[q] != 0.0) atomicAdd(&red[0][c0 + q], nrm[q]);
            if (anr[q] != 0.0) atomicAdd(&red[1][c0 + q], anr[q]);
        }
    }
    __syncthreads();
    if (threadIdx.x < R) {
        const int c = threadIdx.x;
        if (norms && red[0][c] != 0.0) atomicAdd(&norms[f * nstride + ncol0 + c], red[0][c]);
        if (absn && red[1][c] != 0.0) atomicAdd(&absn[f * nstride + ncol0 + c], red[1][c]);
    }
}

template <int R, bool scaled>
void residual_launch_s(const DevModel& m, const double* d_omega, double omega0, int F, const double2* x, int64_t sX,
                       const double2* Fm, int64_t sF, double2* r, int64_t sR, double* norms, int nstride, int c0,
                       double* absn, cudaStream_t st) {
    static const int per_sm = resident_ctas(residual_kernel<R, scaled>);
    const dim3 grid(row_grid_x(m.n, F, per_sm), F);
    residual_kernel<R, scaled><<<grid, kRowThreads, 0, st>>>(m, d_omega, omega0, x ? x + c0 * m.n : nullptr, sX,
                                                             Fm + c0 * m.n, sF, r + c0 * m.n, sR, norms, nstride,
                                                             c0, absn);
}

template <int R>
void residual_launch(const DevModel& m, const double* d_omega, double omega0, int F, const double2* x, int64_t sX,
                     const double2* Fm, int64_t sF, double2* r, int64_t sR, double* norms, int nstride, int c0,
                     bool scaled, double* absn, cudaStream_t st) {
    if (scaled)
        residual_launch_s<R, true>(m, d_omega, omega0, F, x, sX, Fm, sF, r, sR, norms, nstride, c0, absn, st);
    else
        residual_launch_s<R, false>(m, d_omega, omega0, F, x, sX, Fm, sF, r, sR, norms, nstride, c0, absn, st);
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
                     cudaStream_t st, double* absn, int64_t sF) {
    ProfScope ps(PK_RESID, 0.0, st);
    // load columns in power-of-two slices of at most 8
    for (int c0 = 0; c0 < nrhs;) {
        const int left = nrhs - c0;
        const int nc = left >= 8 ? 8 : (left >= 4 ? 4 : (left >= 2 ? 2 : 1));
        switch (nc) {
            case 8: residual_launch<8>(m, d_omega, omega0, F, x, sX, Fm, sF, r, sR, norms, nrhs, c0, scaled, absn, st); break;
            case 4: residual_launch<4>(m, d_omega, omega0, F, x, sX, Fm, sF, r, sR, norms, nrhs, c0, scaled, absn, st); break;
            case 2: residual_launch<2>(m, d_omega, omega0, F, x, sX, Fm, sF, r, sR, norms, nrhs, c0, scaled, absn, st); break;
            default: residual_launch<1>(m, d_omega, omega0, F, x, sX, Fm, sF, r, sR, norms, nrhs, c0, scaled, absn, st);
        }
        c0 += nc;
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
