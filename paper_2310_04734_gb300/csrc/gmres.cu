// GMRES-based iterative refinement (flexible GMRES, right preconditioned by the
// low-precision block-banded factor) for the full-order systems, batched over
// all (frequency, load column) pairs of a sweep batch.
//
// Plain refinement x <- x + LU^-1 r only converges when cond(A) * u_low < 1.
// The thin shell makes the scaled system much worse conditioned at low
// frequencies (cond ~ 1e7 - 1e8 at 20 Hz for the medium model), where FP32
// refinement diverges.  GMRES on the FP64 operator with the FP32 factor as
// preconditioner converges in a few extra iterations there (the paper's
// iterative solver is GMRES, Sec. 3.2; here it refines a direct factor).
//
// Layout: every vector block is [F][nrhs][n] (pair p = f * nrhs + c), the
// Krylov basis V and the preconditioned directions Z are [m+1][F][nrhs][n].
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <complex>
#include <sstream>
#include <string>
#include <vector>

#include "csr_rows.cuh"
#include "engine.h"
#include "prof.h"

namespace fsi {

#define GM_CUDA(call)                                                                                  \
    do {                                                                                               \
        cudaError_t e_ = (call);                                                                       \
        if (e_ != cudaSuccess) {                                                                       \
            std::ostringstream o_;                                                                     \
            o_ << #call << ": " << cudaGetErrorString(e_) << " (" << __FILE__ << ":" << __LINE__ << ")"; \
            set_error(o_.str());                                                                       \
            return FSI_ECUDA;                                                                          \
        }                                                                                              \
    } while (0)

namespace {

constexpr int kGChunks = 32;

inline unsigned cdiv(int64_t a, int64_t b) { return unsigned((a + b - 1) / b); }

constexpr int kApR = 8;    // load columns per thread in the operator application
constexpr int kGrV = 8;    // basis vectors per pass of the Gram kernel
static_assert(kApR == 8, "column slices of 8, 4, 2 and 1");

// w_p = A^ z_p = rs o (A(w_f) (cs o z_p)) for the pairs p = f*nrhs + c0 + c, c < R (a power of
// two), frequency f = blockIdx.y: row groups of kRowLanes lanes form each scaled entry once
// and apply it to the R columns; after the reduce-scatter each lane writes kept_slots<R>
// columns of its row (inactive pairs are not written).
template <int R>
__global__ void __launch_bounds__(kRowThreads) apply_kernel(DevModel m, const double* omega, const double2* z,
                                                            double2* w, int nrhs, int c0, const int32_t* active) {
    constexpr int KS = kept_slots<R>();
    const int f = blockIdx.y;
    const int p0 = f * nrhs + c0;
    bool any = false;
#pragma unroll
    for (int c = 0; c < R; ++c) any = any || !active || active[p0 + c];
    if (!any) return;   // uniform over the CTA
    const double om = omega[f], om2 = om * om, inv_om = 1.0 / om;
    const int g = threadIdx.x & (kRowLanes - 1);
    const int s0 = slot_base<R>(g);
    const bool writer = slot_writer<R>(g);
    for (int64_t base = int64_t(blockIdx.x) * kRowsPerCta; base < m.n; base += int64_t(gridDim.x) * kRowsPerCta) {
        const int64_t i = base + threadIdx.x / kRowLanes;
        const bool valid = i < m.n;
        double2 acc[R];
#pragma unroll
        for (int c = 0; c < R; ++c) acc[c] = make_double2(0.0, 0.0);
        if (valid) {
            const int e1 = __ldg(m.rowptr + i + 1);
            for (int e = __ldg(m.rowptr + i) + g; e < e1; e += kRowLanes) {
                const int64_t col = __ldg(m.col + e);
                double2 a = a_entry_ld(m, e, om, om2);
                const double s = col_scale(m, col, om);
                a.x *= s;
                a.y *= s;
#pragma unroll
                for (int c = 0; c < R; ++c) cfma(acc[c], a, z[int64_t(p0 + c) * m.n + col]);
            }
        }
        group_reduce_scatter<R>(acc, g);
        if (valid && writer) {
            const double rs = row_scale_inv(m, i, inv_om);
#pragma unroll
            for (int q = 0; q < KS; ++q) {
                const int c = s0 + q;
                if (!active || active[p0 + c])
                    w[int64_t(p0 + c) * m.n + i] = make_double2(rs * acc[q].x, rs * acc[q].y);
            }
        }
    }
}

template <int R>
void apply_launch(const DevModel& m, const double* d_omega, const double2* z, double2* w, int nrhs, int c0, int Fb,
                  const int32_t* act, cudaStream_t st) {
    static const int per_sm = resident_ctas(apply_kernel<R>);
    apply_kernel<R><<<dim3(row_grid_x(m.n, Fb, per_sm), Fb), kRowThreads, 0, st>>>(m, d_omega, z, w, nrhs, c0, act);
}

// partial[chunk][p][i0 + i] = sum_{q in chunk} conj(V_{i0+i}[p][q]) w[p][q],  i < NI <= kGrV;
// w is read once per pass for all NI basis vectors (NI a template parameter: a runtime
// count would leave the unused vectors' DFMAs predicated on the FP64 pipe)
template <int NI>
__global__ void bgram_partial_kernel(const double2* V, int64_t sVb, int64_t n, int nv, int i0,
                                     const double2* w, double2* partial, int P, const int32_t* active) {
    constexpr int ni = NI;
    const int p = blockIdx.x, ch = blockIdx.y;
    if (active && !active[p]) return;
    const int64_t len = (n + kGChunks - 1) / kGChunks;
    const int64_t a = ch * len, b = min(n, a + len);
    const double2* wp = w + int64_t(p) * n;
    double2 acc[kGrV];
#pragma unroll
    for (int i = 0; i < kGrV; ++i) acc[i] = make_double2(0.0, 0.0);
    for (int64_t q = a + threadIdx.x; q < b; q += blockDim.x) {
        const double2 wv = wp[q];
#pragma unroll
        for (int i = 0; i < kGrV; ++i)
            if (i < ni) {
                const double2 x = V[int64_t(i0 + i) * sVb + int64_t(p) * n + q];
                cfma(acc[i], make_double2(x.x, -x.y), wv);
            }
    }
    __shared__ double2 red[kGrV][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < kGrV; ++i) {
        if (i >= ni) break;
        double2 v = acc[i];
        for (int off = 16; off > 0; off >>= 1) {
            v.x += __shfl_down_sync(0xffffffffu, v.x, off);
            v.y += __shfl_down_sync(0xffffffffu, v.y, off);
        }
        if (lane == 0) red[i][warp] = v;
    }
    __syncthreads();
    if (threadIdx.x < ni) {
        double2 s2 = make_double2(0.0, 0.0);
        for (int q = 0; q < int(blockDim.x >> 5); ++q) s2 = cadd(s2, red[threadIdx.x][q]);
        partial[(int64_t(ch) * P + p) * nv + i0 + threadIdx.x] = s2;
    }
}

__global__ void bgram_reduce_kernel(const double2* partial, int P, int nv, double2* h) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= P * nv) return;
    double2 s = make_double2(0.0, 0.0);
    for (int ch = 0; ch < kGChunks; ++ch) s = cadd(s, partial[int64_t(ch) * P * nv + q]);
    h[q] = s;
}

void launch_bgram_partial(const double2* V, int64_t sVb, int64_t n, int nv, int i0, int ni, const double2* w,
                          double2* partial, int P, const int32_t* act, cudaStream_t st) {
    const dim3 grid(P, kGChunks);
    switch (ni) {
        case 1: bgram_partial_kernel<1><<<grid, 256, 0, st>>>(V, sVb, n, nv, i0, w, partial, P, act); break;
        case 2: bgram_partial_kernel<2><<<grid, 256, 0, st>>>(V, sVb, n, nv, i0, w, partial, P, act); break;
        case 3: bgram_partial_kernel<3><<<grid, 256, 0, st>>>(V, sVb, n, nv, i0, w, partial, P, act); break;
        case 4: bgram_partial_kernel<4><<<grid, 256, 0, st>>>(V, sVb, n, nv, i0, w, partial, P, act); break;
        case 5: bgram_partial_kernel<5><<<grid, 256, 0, st>>>(V, sVb, n, nv, i0, w, partial, P, act); break;
        case 6: bgram_partial_kernel<6><<<grid, 256, 0, st>>>(V, sVb, n, nv, i0, w, partial, P, act); break;
        case 7: bgram_partial_kernel<7><<<grid, 256, 0, st>>>(V, sVb, n, nv, i0, w, partial, P, act); break;
        default: bgram_partial_kernel<8><<<grid, 256, 0, st>>>(V, sVb, n, nv, i0, w, partial, P, act);
    }
}

// w[p] -= sum_i V_i[p] h[p][i];  also accumulates |w[p]|^2 into nrm[p] (after the update)
__global__ void bupdate_kernel(const double2* V, int64_t sVb, int64_t n, int nv, const double2* h, double2* w,
                               double* nrm, const int32_t* active) {
    const int p = blockIdx.y;
    if (active && !active[p]) return;
    const int64_t q = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    double s2 = 0.0;
    if (q < n) {
        double2 acc = w[int64_t(p) * n + q];
        for (int i = 0; i < nv; ++i) cfms(acc, V[int64_t(i) * sVb + int64_t(p) * n + q], h[int64_t(p) * nv + i]);
        w[int64_t(p) * n + q] = acc;
        s2 = acc.x * acc.x + acc.y * acc.y;
    }
    for (int off = 16; off > 0; off >>= 1) s2 += __shfl_down_sync(0xffffffffu, s2, off);
    if ((threadIdx.x & 31) == 0 && s2 != 0.0) atomicAdd(&nrm[p], s2);
}

// dst[p] = src[p] * scale[p]
__global__ void bscale_kernel(const double2* src, double2* dst, const double* scale, int64_t n,
                              const int32_t* active) {
    const int p = blockIdx.y;
    if (active && !active[p]) return;
    const int64_t q = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const double s = scale[p];
    const double2 v = src[int64_t(p) * n + q];
    dst[int64_t(p) * n + q] = make_double2(s * v.x, s * v.y);
}

// x[p] += sum_j Z_j[p] y[p][j]
__global__ void bcombine_kernel(const double2* Z, int64_t sZb, int64_t n, int nj, const double2* y, double2* x) {
    const int p = blockIdx.y;
    const int64_t q = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (q >= n) return;
    double2 acc = x[int64_t(p) * n + q];
    for (int j = 0; j < nj; ++j) {
        const double2 c = y[int64_t(p) * nj + j];
        if (c.x != 0.0 || c.y != 0.0) cfma(acc, Z[int64_t(j) * sZb + int64_t(p) * n + q], c);
    }
    x[int64_t(p) * n + q] = acc;
}

template <typename T2>
__global__ void to_low_unit_kernel(const double2* v, T2* y, int64_t cnt) {
    using R = decltype(T2::x);
    const int64_t q = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (q >= cnt) return;
    y[q] = mk<T2>(R(v[q].x), R(v[q].y));
}

template <typename T2>
__global__ void to_high_kernel(const T2* y, double2* v, int64_t cnt) {
    const int64_t q = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (q >= cnt) return;
    v[q] = make_double2(double(y[q].x), double(y[q].y));
}

using cd = std::complex<double>;

}  // namespace

size_t gmres_ws_bytes(int64_t n, int P, int m) {
    Carver c(nullptr, 0);
    c.take<double2>(size_t(m + 1) * P * n);   // V
    c.take<double2>(size_t(m) * P * n);       // Z
    c.take<double2>(size_t(P) * n);           // w
    c.take<double2>(size_t(kGChunks) * P * (m + 1));
    c.take<double2>(size_t(P) * (m + 1));     // h
    c.take<double2>(size_t(P) * m);           // y
    c.take<double>(P);                        // nrm
    c.take<double>(P);                        // scale
    c.take<int32_t>(P);                       // active
    c.take<int32_t>(P);                       // frequencies with an active pair
    return align_up(c.used);
}

template <typename R>
fsi_status fgmres_solve(const DevModel& m, Factor<R>& fc, int Fb, const double* d_omega, const double2* Bdev,
                        int nrhs, double2* xhat, double2* rhat, typename Cplx<R>::T* y, double* norms, double* fnorms,
                        double* absn, int64_t sV, int restart, int max_cycles, double tol, void* gws, size_t gws_bytes,
                        std::vector<int>& it_done, std::vector<double>& rel, cudaStream_t st) {
    using T2 = typename Cplx<R>::T;
    const int64_t n = m.n;
    const int P = Fb * nrhs;
    const int mm = std::max(1, restart);
    Carver c(gws, gws_bytes);
    double2* V = c.take<double2>(size_t(mm + 1) * P * n);
    double2* Z = c.take<double2>(size_t(mm) * P * n);
    double2* w = c.take<double2>(size_t(P) * n);
    double2* part = c.take<double2>(size_t(kGChunks) * P * (mm + 1));
    double2* yd = c.take<double2>(size_t(P) * mm);
    double* nrm = c.take<double>(P);
    double* scl = c.take<double>(P);
    int32_t* act = c.take<int32_t>(P);
    int32_t* flist = c.take<int32_t>(P);
    if (!c.fits()) {
        set_error("GMRES workspace too small");
        return FSI_ENOMEM;
    }
    const int64_t sVb = int64_t(P) * n;   // stride between basis vectors
    (void)sV;
    std::vector<double> hf(P), hn(P), hs(P), ha(P);
    std::vector<double> flo(P, 0.0);   // relative rounding floor of the last explicit residual
    std::vector<int32_t> hact(P);
    std::vector<int32_t> hfl;
    hfl.reserve(Fb);
    // r = R f, |R f|
    GM_CUDA(cudaMemsetAsync(fnorms, 0, sizeof(double) * P, st));
    launch_residual(m, d_omega, 0.0, Fb, nullptr, int64_t(nrhs) * n, Bdev, nrhs, rhat, int64_t(nrhs) * n, fnorms,
                    true, st);
    GM_CUDA(cudaMemcpyAsync(hf.data(), fnorms, sizeof(double) * P, cudaMemcpyDeviceToHost, st));
    GM_CUDA(cudaMemsetAsync(xhat, 0, sizeof(double2) * P * n, st));
    GM_CUDA(cudaMemcpyAsync(hn.data(), fnorms, sizeof(double) * P, cudaMemcpyDeviceToHost, st));
    GM_CUDA(cudaStreamSynchronize(st));
    std::vector<int> pdone(P, -1), inner_done(P, -1);
    int total_it = 0;
    std::vector<double> prel(P, 1.0);
    for (int p = 0; p < P; ++p) prel[p] = hf[p] > 0 ? std::sqrt(hn[p] / hf[p]) : 0.0;
    auto conv = [&](int p) { return prel[p] <= std::max(tol, flo[p]); };
    for (int cyc = 0; cyc < max_cycles; ++cyc) {
        // active pairs: not yet at tol
        int nact = 0;
        for (int p = 0; p < P; ++p) {
            hact[p] = conv(p) ? 0 : 1;
            if (!hact[p] && pdone[p] < 0) pdone[p] = inner_done[p] >= 0 ? inner_done[p] : total_it;
            nact += hact[p];
        }
        if (nact == 0) break;
        GM_CUDA(cudaMemcpyAsync(act, hact.data(), sizeof(int32_t) * P, cudaMemcpyHostToDevice, st));
        // v_0 = r / beta
        std::vector<double> beta(P);
        for (int p = 0; p < P; ++p) {
            beta[p] = std::sqrt(hn[p]);
            hs[p] = beta[p] > 0 ? 1.0 / beta[p] : 0.0;
        }
        GM_CUDA(cudaMemcpyAsync(scl, hs.data(), sizeof(double) * P, cudaMemcpyHostToDevice, st));
        bscale_kernel<<<dim3(cdiv(n, 256), P), 256, 0, st>>>(rhat, V, scl, n, nullptr);
        // Givens state per pair
        std::vector<std::vector<cd>> H(P, std::vector<cd>(size_t(mm + 1) * mm, cd(0, 0)));
        std::vector<std::vector<cd>> g(P, std::vector<cd>(mm + 1, cd(0, 0)));
        std::vector<std::vector<double>> cs(P, std::vector<double>(mm, 0.0));
        std::vector<std::vector<cd>> sn(P, std::vector<cd>(mm, cd(0, 0)));
        std::vector<int> kdim(P, 0);
        std::vector<int32_t> live = hact;
        for (int p = 0; p < P; ++p) g[p][0] = cd(beta[p], 0.0);
        std::vector<double2> hbuf(size_t(P) * (mm + 1));
        int j = 0;
        for (; j < mm; ++j) {
            // z_j = M^-1 v_j (low precision), back to FP64
            to_low_unit_kernel<T2><<<cdiv(int64_t(P) * n, 256), 256, 0, st>>>(V + int64_t(j) * sVb, y, int64_t(P) * n);
            // solve only the frequencies that still have a live pair
            hfl.clear();
            for (int f = 0; f < Fb; ++f) {
                bool any_live = false;
                for (int cc = 0; cc < nrhs; ++cc) any_live = any_live || live[f * nrhs + cc];
                if (any_live) hfl.push_back(f);
            }
            const bool sub = int(hfl.size()) < Fb;
            if (sub)
                GM_CUDA(cudaMemcpyAsync(flist, hfl.data(), sizeof(int32_t) * hfl.size(), cudaMemcpyHostToDevice, st));
            fsi_status s = solve_batch<R>(m, fc, Fb, y, int64_t(nrhs) * n, nrhs, st, sub ? flist : nullptr,
                                          int(hfl.size()));
            if (s != FSI_OK) return s;
            to_high_kernel<T2><<<cdiv(int64_t(P) * n, 256), 256, 0, st>>>(y, Z + int64_t(j) * sVb, int64_t(P) * n);
            {
                ProfScope ps(PK_RESID, 0.0, st);
                const double2* zj = Z + int64_t(j) * sVb;
                // load columns in power-of-two slices of at most kApR
                for (int c0 = 0; c0 < nrhs;) {
                    const int left = nrhs - c0;
                    const int nc = left >= 8 ? 8 : (left >= 4 ? 4 : (left >= 2 ? 2 : 1));
                    switch (nc) {
                        case 8: apply_launch<8>(m, d_omega, zj, w, nrhs, c0, Fb, act, st); break;
                        case 4: apply_launch<4>(m, d_omega, zj, w, nrhs, c0, Fb, act, st); break;
                        case 2: apply_launch<2>(m, d_omega, zj, w, nrhs, c0, Fb, act, st); break;
                        default: apply_launch<1>(m, d_omega, zj, w, nrhs, c0, Fb, act, st);
                    }
                    c0 += nc;
                }
            }
            // CGS2 against v_0..v_j
            for (int pass = 0; pass < 2; ++pass) {
                ProfScope ps(PK_RESID, 0.0, st);
                for (int i0 = 0; i0 <= j; i0 += kGrV)
                    launch_bgram_partial(V, sVb, n, j + 1, i0, std::min(kGrV, j + 1 - i0), w, part, P, act, st);
                bgram_reduce_kernel<<<cdiv(int64_t(P) * (j + 1), 256), 256, 0, st>>>(part, P, j + 1, yd);
                GM_CUDA(cudaMemsetAsync(nrm, 0, sizeof(double) * P, st));
                bupdate_kernel<<<dim3(cdiv(n, 256), P), 256, 0, st>>>(V, sVb, n, j + 1, yd, w, nrm, act);
                GM_CUDA(cudaMemcpyAsync(hbuf.data(), yd, sizeof(double2) * P * (j + 1),
                                        cudaMemcpyDeviceToHost, st));
                GM_CUDA(cudaStreamSynchronize(st));
                for (int p = 0; p < P; ++p)
                    for (int i = 0; i <= j; ++i)
                        H[p][size_t(i) * mm + j] += cd(hbuf[size_t(p) * (j + 1) + i].x, hbuf[size_t(p) * (j + 1) + i].y);
            }
            GM_CUDA(cudaMemcpyAsync(hn.data(), nrm, sizeof(double) * P, cudaMemcpyDeviceToHost, st));
            GM_CUDA(cudaStreamSynchronize(st));
            ++total_it;
            bool any = false;
            for (int p = 0; p < P; ++p) {
                if (!live[p]) {
                    hs[p] = 0.0;
                    continue;
                }
                const double hj1 = std::sqrt(hn[p]);
                H[p][size_t(j + 1) * mm + j] = cd(hj1, 0.0);
                hs[p] = hj1 > 0 ? 1.0 / hj1 : 0.0;
                // apply previous rotations to column j
                for (int i = 0; i < j; ++i) {
                    const cd a = H[p][size_t(i) * mm + j], b = H[p][size_t(i + 1) * mm + j];
                    H[p][size_t(i) * mm + j] = cs[p][i] * a + sn[p][i] * b;
                    H[p][size_t(i + 1) * mm + j] = -std::conj(sn[p][i]) * a + cs[p][i] * b;
                }
                const cd a = H[p][size_t(j) * mm + j], b = H[p][size_t(j + 1) * mm + j];
                const double den = std::sqrt(std::norm(a) + std::norm(b));
                double cc = 1.0;
                cd ss(0, 0);
                if (den > 0) {
                    if (std::abs(a) == 0.0) {
                        cc = 0.0;
                        ss = std::conj(b) / std::abs(b);
                    } else {
                        cc = std::abs(a) / den;
                        ss = (a / std::abs(a)) * std::conj(b) / den;
                    }
                }
                cs[p][j] = cc;
                sn[p][j] = ss;
                H[p][size_t(j) * mm + j] = cc * a + ss * b;
                H[p][size_t(j + 1) * mm + j] = cd(0, 0);
                g[p][j + 1] = -std::conj(ss) * g[p][j];
                g[p][j] = cc * g[p][j];
                kdim[p] = j + 1;
                const double est = std::abs(g[p][j + 1]) / std::sqrt(hf[p]);
                if (est <= 0.5 * std::max(tol, flo[p]) || hj1 == 0.0) {
                    live[p] = 0;
                    if (inner_done[p] < 0) inner_done[p] = total_it;
                } else {
                    any = true;
                }
            }
            if (!any || j + 1 == mm) {
                ++j;
                break;
            }
            GM_CUDA(cudaMemcpyAsync(scl, hs.data(), sizeof(double) * P, cudaMemcpyHostToDevice, st));
            std::vector<int32_t> lv = live;
            GM_CUDA(cudaMemcpyAsync(act, lv.data(), sizeof(int32_t) * P, cudaMemcpyHostToDevice, st));
            bscale_kernel<<<dim3(cdiv(n, 256), P), 256, 0, st>>>(w, V + int64_t(j + 1) * sVb, scl, n, act);
            GM_CUDA(cudaStreamSynchronize(st));
        }
        // solve the triangular systems and combine x += Z y
        const int nj = j;
        std::vector<double2> yh(size_t(P) * nj, make_double2(0, 0));
        for (int p = 0; p < P; ++p) {
            const int kd = hact[p] ? kdim[p] : 0;
            std::vector<cd> yy(nj, cd(0, 0));
            for (int i = kd - 1; i >= 0; --i) {
                cd s = g[p][i];
                for (int q = i + 1; q < kd; ++q) s -= H[p][size_t(i) * mm + q] * yy[q];
                yy[i] = s / H[p][size_t(i) * mm + i];
            }
            for (int i = 0; i < nj; ++i) yh[size_t(p) * nj + i] = make_double2(yy[i].real(), yy[i].imag());
        }
        GM_CUDA(cudaMemcpyAsync(yd, yh.data(), sizeof(double2) * P * nj, cudaMemcpyHostToDevice, st));
        bcombine_kernel<<<dim3(cdiv(n, 256), P), 256, 0, st>>>(Z, sVb, n, nj, yd, xhat);
        // explicit residual
        GM_CUDA(cudaMemsetAsync(norms, 0, sizeof(double) * P, st));
        GM_CUDA(cudaMemsetAsync(absn, 0, sizeof(double) * P, st));
        launch_residual(m, d_omega, 0.0, Fb, xhat, int64_t(nrhs) * n, Bdev, nrhs, rhat, int64_t(nrhs) * n, norms,
                        true, st, absn);
        GM_CUDA(cudaMemcpyAsync(hn.data(), norms, sizeof(double) * P, cudaMemcpyDeviceToHost, st));
        GM_CUDA(cudaMemcpyAsync(ha.data(), absn, sizeof(double) * P, cudaMemcpyDeviceToHost, st));
        GM_CUDA(cudaStreamSynchronize(st));
        for (int p = 0; p < P; ++p) {
            prel[p] = hf[p] > 0 ? std::sqrt(hn[p] / hf[p]) : 0.0;
            flo[p] = hf[p] > 0 ? kResFloor * std::sqrt(ha[p] / hf[p]) : 0.0;
            if (!conv(p)) inner_done[p] = -1;   // the estimate was optimistic: keep iterating
        }
    }
    for (int p = 0; p < P; ++p)
        if (pdone[p] < 0 && conv(p)) pdone[p] = inner_done[p] >= 0 ? inner_done[p] : total_it;
    it_done.assign(Fb, -1);
    rel.assign(Fb, 0.0);
    for (int f = 0; f < Fb; ++f) {
        int it = 0;
        bool ok = true;
        double r = 0.0;
        for (int cc = 0; cc < nrhs; ++cc) {
            const int p = f * nrhs + cc;
            r = std::max(r, prel[p]);
            if (!conv(p)) ok = false;
            it = std::max(it, pdone[p] < 0 ? total_it : std::max(pdone[p], 1));   // solves until this pair converged
        }
        rel[f] = r;
        it_done[f] = ok ? it : -1;
    }
    GM_CUDA(cudaGetLastError());
    return FSI_OK;
}

template fsi_status fgmres_solve<float>(const DevModel&, Factor<float>&, int, const double*, const double2*, int,
                                        double2*, double2*, float2*, double*, double*, double*, int64_t, int, int, double,
                                        void*, size_t, std::vector<int>&, std::vector<double>&, cudaStream_t);
template fsi_status fgmres_solve<double>(const DevModel&, Factor<double>&, int, const double*, const double2*, int,
                                         double2*, double2*, double2*, double*, double*, double*, int64_t, int, int, double,
                                         void*, size_t, std::vector<int>&, std::vector<double>&, cudaStream_t);

}  // namespace fsi
