// Greedy choice of rational Arnoldi expansion points (paper Sec. 3.3: the
// expansion points are added where the reduced model's error is largest; the
// paper measures that error against full-order solutions and notes that a
// cheaper estimate can replace it, Sec. 5).
//
// Estimate: the relative residual of the equilibrated full-order system,
//   est(w) = |R(w) (F - A(w) V x_R(w))|_F / |R(w) F|_F ,
// R(w) the row scaling of the full-order sweep.  It is evaluated exactly,
// without forming V x_R, from Gram blocks of Y = [K V, D V, M V]:
// A(w) V x_R = Y z with z = [x_R; i w x_R; -w^2 x_R] (interleaved per basis
// column), and R(w)^2 = W_s + W_f / w^2 with fixed diagonal weights on the
// shell rows (1/|K_ii|) and the fluid rows (1/(rho |K_ii|)), so
//   |R r|^2 = sum_{sel in s,f} c_sel(w) (F^H W F - 2 Re(h^H z) + z^H G z),
//   G = Y^H W Y (3k x 3k), h = Y^H W F.
// The Gram blocks grow with the basis: only the rows/columns of new basis
// vectors are computed after each expansion point.  The difference of large
// terms limits the estimate's relative accuracy to about u / est^2, which is
// ample above est ~ 1e-7.
//
// Loop: start from the given points (or the middle candidate), build the basis,
// project, estimate on every candidate, stop when the largest estimate is
// <= tol, at max_shifts points or at kmax columns; otherwise add the candidate
// of largest estimate (ties: lowest frequency) that is more than one grid step
// away from every existing point, extend the basis with its moments and repeat.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <numeric>
#include <sstream>
#include <string>
#include <vector>

#include "csr_rows.cuh"
#include "engine.h"
#include "fsi_internal.h"
#include "kernels.cuh"
#include "rom_internal.h"

namespace fsi {

#define GR_CUDA(call)                                                                                  \
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

constexpr int kWSplit = 16;     // split over rows of the Gram products
constexpr int kCandBatch = 128;  // candidate frequencies per reduced-solve batch

inline unsigned cdiv(int64_t a, int64_t b) { return unsigned((a + b - 1) / b); }

// Estimator features of candidate i: position in the band, distances to the three nearest
// expansion points (band-relative, 1 when missing), log10 of the residual estimate / 4.
void features(const double* cand, int ncand, const double* shifts, int nshift, const double* est, double lo,
              double hi, float* X) {
    const double span = hi > lo ? hi - lo : 1.0;
    std::vector<double> d(nshift);
    for (int i = 0; i < ncand; ++i) {
        for (int j = 0; j < nshift; ++j) d[j] = std::fabs(cand[i] - shifts[j]) / span;
        std::sort(d.begin(), d.end());
        float* x = X + int64_t(i) * 5;
        x[0] = float((cand[i] - lo) / span);
        for (int j = 0; j < 3; ++j) x[1 + j] = float(j < nshift ? std::min(d[j], 1.0) : 1.0);
        x[4] = float(std::log10(std::max(est[i], 1e-16)) / 4.0);
    }
}

// weight of row i: 1 (sel 0); on the fluid rows 1/(rho |K_ii|) (sel 1); on the shell rows 1/|K_ii| (sel 2)
__device__ __forceinline__ double row_weight(const DevModel& m, int64_t i, int sel) {
    if (sel == 0) return 1.0;
    const bool fl = is_fluid(m, i);
    if ((sel == 1) != fl) return 0.0;
    const double kd = m.kdiag[i];
    return fl ? 1.0 / (m.rho * kd) : 1.0 / kd;
}

// Y[:, 3j + w] = A_w V[:, j] for j in [j0, j0 + nj), A_0 = K, A_1 = D, A_2 = M (one pass over
// each row, j = j0 + blockIdx.y); row groups of kRowLanes lanes, lanes 0..2 of a group write
__global__ void __launch_bounds__(kRowThreads) yspmm_kernel(DevModel m, const double2* V, int j0, double2* Y) {
    const int j = j0 + blockIdx.y;
    const int g = threadIdx.x & (kRowLanes - 1);
    const double2* vj = V + int64_t(j) * m.n;
    for (int64_t base = int64_t(blockIdx.x) * kRowsPerCta; base < m.n; base += int64_t(gridDim.x) * kRowsPerCta) {
        const int64_t i = base + threadIdx.x / kRowLanes;
        const bool valid = i < m.n;
        double2 y[4] = {make_double2(0.0, 0.0), make_double2(0.0, 0.0), make_double2(0.0, 0.0),
                        make_double2(0.0, 0.0)};   // slot 3 unused (power-of-two reduce-scatter)
        if (valid) {
            const int e1 = __ldg(m.rowptr + i + 1);
            for (int e = __ldg(m.rowptr + i) + g; e < e1; e += kRowLanes) {
                const double2 x = vj[__ldg(m.col + e)];
                cfma(y[0], __ldg(m.K + e), x);
                cfma(y[1], __ldg(m.D + e), x);
                const double mm = __ldg(m.M + e);
                y[2].x = fma(mm, x.x, y[2].x);
                y[2].y = fma(mm, x.y, y[2].y);
            }
        }
        group_reduce_scatter<4>(y, g);   // lane g now holds slot g (kRowLanes = 4)
        if (valid && g < 3) Y[(int64_t(3) * j + g) * m.n + i] = y[0];
    }
}

// partial[s][b][a] = sum_{i in split s} w(i) conj(A[i][a0 + a]) B[i][b0 + b]   (32 x 32 output tiles)
__global__ void __launch_bounds__(256) wgram_partial_kernel(DevModel m, int sel, const double2* A, int a0, int na,
                                                            const double2* B, int b0, int nb, double2* partial) {
    __shared__ double2 As[32][33];
    __shared__ double2 Bs[32][33];
    const int ta = blockIdx.x, tb = blockIdx.y, s = blockIdx.z;
    const int64_t n = m.n;
    const int64_t len = (n + kWSplit - 1) / kWSplit;
    const int64_t i0 = s * len, i1 = min(n, i0 + len);
    const int tid = threadIdx.x;
    const int ra = tid >> 3;          // output row within the tile
    const int cb = (tid & 7) * 4;     // four output columns
    double2 acc[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[q] = make_double2(0.0, 0.0);
    for (int64_t base = i0; base < i1; base += 32) {
        for (int idx = tid; idx < 32 * 32; idx += 256) {
            const int col = idx >> 5, ii = idx & 31;
            const int64_t gi = base + ii;
            const int ja = ta * 32 + col, jb = tb * 32 + col;
            double2 av = make_double2(0.0, 0.0), bv = av;
            if (gi < i1) {
                const double wgt = row_weight(m, gi, sel);
                if (ja < na) {
                    av = A[int64_t(a0 + ja) * n + gi];
                    av = make_double2(wgt * av.x, -wgt * av.y);   // w conj(a)
                }
                if (jb < nb) bv = B[int64_t(b0 + jb) * n + gi];
            }
            As[ii][col] = av;
            Bs[ii][col] = bv;
        }
        __syncthreads();
#pragma unroll 8
        for (int ii = 0; ii < 32; ++ii) {
            const double2 a = As[ii][ra];
#pragma unroll
            for (int q = 0; q < 4; ++q) cfma(acc[q], a, Bs[ii][cb + q]);
        }
        __syncthreads();
    }
    const int a = ta * 32 + ra;
    if (a >= na) return;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int b = tb * 32 + cb + q;
        if (b < nb) partial[(int64_t(s) * nb + b) * na + a] = acc[q];
    }
}

// C[(cb0 + b) * ldc + ca0 + a] = sum_s partial; with mirror, also C[(ca0 + a) * ldc + cb0 + b] = conj(.)
// for the entries with ca0 + a < mirror_below (the old-by-new block of a Hermitian product)
__global__ void wgram_reduce_kernel(const double2* partial, int na, int nb, double2* C, int64_t ldc, int ca0, int cb0,
                                    int mirror_below) {
    const int64_t q = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (q >= int64_t(na) * nb) return;
    const int b = int(q / na), a = int(q - int64_t(b) * na);
    double2 s = make_double2(0.0, 0.0);
    for (int p = 0; p < kWSplit; ++p) s = cadd(s, partial[int64_t(p) * na * nb + q]);
    C[int64_t(cb0 + b) * ldc + ca0 + a] = s;
    if (ca0 + a < mirror_below) C[int64_t(ca0 + a) * ldc + cb0 + b] = make_double2(s.x, -s.y);
}

// K_R, D_R, M_R (k x k, ld k) from P = V^H Y (ld kmax); f_R (k x nrhs, ld k) from Pf (ld kmax)
__global__ void extract_reduced_kernel(const double2* P, int64_t ldp, const double2* Pf, int k, int nrhs,
                                       double2* KR, double2* DR, double2* MR, double2* fR) {
    const int64_t q = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (q < int64_t(k) * k) {
        const int j = int(q / k), a = int(q - int64_t(j) * k);
        KR[q] = P[int64_t(3 * j + 0) * ldp + a];
        DR[q] = P[int64_t(3 * j + 1) * ldp + a];
        MR[q] = P[int64_t(3 * j + 2) * ldp + a];
    }
    if (q < int64_t(k) * nrhs) {
        const int c = int(q / k), a = int(q - int64_t(c) * k);
        fR[q] = Pf[int64_t(c) * ldp + a];
    }
}

// One CTA per (load column c, frequency f) of a reduced batch: num = |R r|^2, den = |R F|^2
__global__ void proxy_kernel(const double2* G, const double* cs, const double* omega, int k, int nrhs,
                             const double2* Gf, const double2* Gs, int64_t ldg, const double2* Hf, const double2* Hs,
                             int64_t ldh, const double* fnf, const double* fns, double* num, double* den) {
    extern __shared__ double2 z[];   // 3k
    const int c = blockIdx.x, f = blockIdx.y;
    const int ld = k + nrhs;
    const double w = omega[f];
    for (int j = threadIdx.x; j < k; j += blockDim.x) {
        const double2 y = G[int64_t(f) * k * ld + int64_t(j) * ld + k + c];
        const double s = cs[int64_t(f) * k + j];
        const double2 x = make_double2(s * y.x, s * y.y);
        z[3 * j + 0] = x;
        z[3 * j + 1] = make_double2(-w * x.y, w * x.x);
        z[3 * j + 2] = make_double2(-w * w * x.x, -w * w * x.y);
    }
    __syncthreads();
    const int K3 = 3 * k;
    double qf = 0.0, qs = 0.0, lf = 0.0, ls = 0.0;
    for (int a = threadIdx.x; a < K3; a += blockDim.x) {
        double2 gf = make_double2(0.0, 0.0), gs = gf;
        for (int b = 0; b < K3; ++b) {
            const double2 zb = z[b];
            cfma(gf, Gf[int64_t(b) * ldg + a], zb);
            cfma(gs, Gs[int64_t(b) * ldg + a], zb);
        }
        const double2 za = z[a];
        qf += za.x * gf.x + za.y * gf.y;   // Re(conj(z_a) (G z)_a)
        qs += za.x * gs.x + za.y * gs.y;
        const double2 hf = Hf[int64_t(c) * ldh + a], hs = Hs[int64_t(c) * ldh + a];
        lf += hf.x * za.x + hf.y * za.y;   // Re(conj(h_a) z_a)
        ls += hs.x * za.x + hs.y * za.y;
    }
    __shared__ double red[4][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int off = 16; off > 0; off >>= 1) {
        qf += __shfl_down_sync(0xffffffffu, qf, off);
        qs += __shfl_down_sync(0xffffffffu, qs, off);
        lf += __shfl_down_sync(0xffffffffu, lf, off);
        ls += __shfl_down_sync(0xffffffffu, ls, off);
    }
    if (lane == 0) {
        red[0][warp] = qf;
        red[1][warp] = qs;
        red[2][warp] = lf;
        red[3][warp] = ls;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t[4] = {0, 0, 0, 0};
        for (int q = 0; q < int(blockDim.x >> 5); ++q)
            for (int u = 0; u < 4; ++u) t[u] += red[u][q];
        const double rf = fnf[c] - 2.0 * t[2] + t[0];
        const double rsh = fns[c] - 2.0 * t[3] + t[1];
        const double iw2 = 1.0 / (w * w);
        num[int64_t(f) * nrhs + c] = rsh + rf * iw2;
        den[int64_t(f) * nrhs + c] = fns[c] + fnf[c] * iw2;
    }
}

__global__ void gather_rows_kernel(const double2* V, int64_t n, int k, const int32_t* rcv, int nrcv, double2* CR) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= k * nrcv) return;
    const int j = q / nrcv, ir = q - j * nrcv;
    CR[q] = V[int64_t(j) * n + rcv[ir]];   // column-major nrcv x k
}

struct GreedyWS {
    void* build = nullptr;
    size_t build_bytes = 0;
    double2 *Y, *P, *Pf, *Gf, *Gs, *Hf, *Hs, *part;
    double *fnf, *fns, *num, *den;
    float *xf = nullptr, *yf = nullptr;   // estimator features / predictions of one candidate batch
    void* rws = nullptr;
    size_t rws_bytes = 0;
    int64_t ldp = 0, ldg = 0;
    size_t part_elems = 0;

    template <typename R>
    void carve(Carver& c, const fsi_dims& d, int nrhs, const fsi_greedy_opts& o) {
        const int64_t n = d.n;
        const int K = o.kmax;
        build_bytes = rom_build_ws<R>(d, nrhs, o.q, K, o.build);
        build = c.take<char>(build_bytes);
        ldp = K;
        ldg = 3 * int64_t(K);
        Y = c.take<double2>(size_t(n) * 3 * K);
        P = c.take<double2>(size_t(K) * 3 * K);
        Pf = c.take<double2>(size_t(K) * nrhs);
        Gf = c.take<double2>(size_t(ldg) * ldg);
        Gs = c.take<double2>(size_t(ldg) * ldg);
        Hf = c.take<double2>(size_t(ldg) * nrhs);
        Hs = c.take<double2>(size_t(ldg) * nrhs);
        part_elems = size_t(kWSplit) * ldg * ldg;
        part = c.take<double2>(part_elems);
        fnf = c.take<double>(nrhs);
        fns = c.take<double>(nrhs);
        num = c.take<double>(size_t(kCandBatch) * nrhs);
        den = c.take<double>(size_t(kCandBatch) * nrhs);
        rws_bytes = reduced_solve_ws(K, nrhs, kCandBatch);
        rws = c.take<char>(rws_bytes);
        xf = c.take<float>(size_t(kCandBatch) * 5);
        yf = c.take<float>(kCandBatch);
    }
};

// C(block) = A[:, a0:a0+na]^H W_sel B[:, b0:b0+nb] into C at (ca0, cb0)
fsi_status wgram(const DevModel& m, int sel, const double2* A, int a0, int na, const double2* B, int b0, int nb,
                 double2* part, double2* C, int64_t ldc, int ca0, int cb0, int mirror_below, cudaStream_t st) {
    if (na <= 0 || nb <= 0) return FSI_OK;
    wgram_partial_kernel<<<dim3(cdiv(na, 32), cdiv(nb, 32), kWSplit), 256, 0, st>>>(m, sel, A, a0, na, B, b0, nb,
                                                                                   part);
    wgram_reduce_kernel<<<cdiv(int64_t(na) * nb, 256), 256, 0, st>>>(part, na, nb, C, ldc, ca0, cb0, mirror_below);
    GR_CUDA(cudaGetLastError());
    return FSI_OK;
}

// Gram blocks for basis columns [k0, k1) (the first k0 are already in place)
fsi_status grow_gram(const DevModel& m, GreedyWS& w, const double2* V, const double2* F, int nrhs, int k0, int k1,
                     cudaStream_t st) {
    if (k1 <= k0) return FSI_OK;
    const int64_t n = m.n;
    static const int per_sm = resident_ctas(yspmm_kernel);
    yspmm_kernel<<<dim3(row_grid_x(n, k1 - k0, per_sm), k1 - k0), kRowThreads, 0, st>>>(m, V, k0, w.Y);
    GR_CUDA(cudaGetLastError());
    // P = V^H Y: new columns of Y against all of V, and new rows of V against the old columns of Y
    fsi_status s = wgram(m, 0, V, 0, k1, w.Y, 3 * k0, 3 * (k1 - k0), w.part, w.P, w.ldp, 0, 3 * k0, 0, st);
    if (s == FSI_OK) s = wgram(m, 0, V, k0, k1 - k0, w.Y, 0, 3 * k0, w.part, w.P, w.ldp, k0, 0, 0, st);
    // f_R rows of the new columns
    if (s == FSI_OK) s = wgram(m, 0, V, k0, k1 - k0, F, 0, nrhs, w.part, w.Pf, w.ldp, k0, 0, 0, st);
    // weighted Gram blocks of Y (Hermitian: compute the new columns, mirror the old-by-new block)
    for (int sel = 1; sel <= 2 && s == FSI_OK; ++sel) {
        double2* G = sel == 1 ? w.Gf : w.Gs;
        double2* H = sel == 1 ? w.Hf : w.Hs;
        s = wgram(m, sel, w.Y, 0, 3 * k1, w.Y, 3 * k0, 3 * (k1 - k0), w.part, G, w.ldg, 0, 3 * k0, 3 * k0, st);
        if (s == FSI_OK) s = wgram(m, sel, w.Y, 3 * k0, 3 * (k1 - k0), F, 0, nrhs, w.part, H, w.ldg, 3 * k0, 0, 0, st);
    }
    return s;
}

template <typename R>
fsi_status run_greedy(const fsi_dims& d, const void* d_model, const double2* F, int nrhs, const double* cand,
                      int ncand, const double* init_hz, int ninit, const fsi_greedy_opts& o, void* ws, size_t ws_bytes,
                      double2* V, int* k_out, double2* KR, double2* DR, double2* MR, double2* fR, const int32_t* rcv,
                      int nrcv, double2* CR, double* shifts_out, int* nshift_out, double* est_out, double* hist_out,
                      cudaStream_t st, int k_seed = 0, const double* seed_hz = nullptr, int nseed = 0,
                      MomentStore* store = nullptr) {
    Carver c(ws, ws_bytes);
    GreedyWS w;
    w.carve<R>(c, d, nrhs, o);
    if (!c.fits()) {
        set_error("rom_greedy workspace too small: need " + std::to_string(align_up(c.used)) + " bytes");
        return FSI_ENOMEM;
    }
    const DevModel m = dev_model(d, d_model);
    // |W_sel^1/2 F|^2 per load column
    {
        fsi_status s = FSI_OK;
        double2* tmp = w.Hf;   // nrhs x nrhs scratch before the first use of Hf
        std::vector<double2> h(size_t(nrhs) * nrhs);
        std::vector<double> fn(nrhs);
        for (int sel = 1; sel <= 2; ++sel) {
            s = wgram(m, sel, F, 0, nrhs, F, 0, nrhs, w.part, tmp, nrhs, 0, 0, 0, st);
            if (s != FSI_OK) return s;
            GR_CUDA(cudaMemcpyAsync(h.data(), tmp, sizeof(double2) * nrhs * nrhs, cudaMemcpyDeviceToHost, st));
            GR_CUDA(cudaStreamSynchronize(st));
            for (int cc = 0; cc < nrhs; ++cc) fn[cc] = h[size_t(cc) * nrhs + cc].x;
            GR_CUDA(cudaMemcpyAsync(sel == 1 ? w.fnf : w.fns, fn.data(), sizeof(double) * nrhs,
                                    cudaMemcpyHostToDevice, st));
        }
        GR_CUDA(cudaStreamSynchronize(st));
    }
    const double step = ncand > 1 ? [&] {
        double mn = INFINITY;
        for (int i = 1; i < ncand; ++i) mn = std::min(mn, cand[i] - cand[i - 1]);
        return mn;
    }()
                                  : 0.0;
    // expansion points whose moments V already holds (k_seed columns), then the fresh initial points
    std::vector<double> shifts(seed_hz, seed_hz + nseed), fresh;
    if (ninit > 0)
        fresh.assign(init_hz, init_hz + ninit);
    else if (nseed == 0)
        fresh.push_back(cand[ncand / 2]);
    if (int(shifts.size() + fresh.size()) > o.max_shifts) fresh.resize(std::max(0, o.max_shifts - nseed));
    int k = k_seed, k1 = k_seed;
    fsi_status s = FSI_OK;
    if (!fresh.empty()) {
        s = rom_build_append<R>(d, d_model, fresh.data(), int(fresh.size()), o.q, F, nrhs, o.kmax, o.build, w.build,
                                w.build_bytes, V, k_seed, &k1, st, store);
        if (s != FSI_OK) return s;
        shifts.insert(shifts.end(), fresh.begin(), fresh.end());
    }
    s = grow_gram(m, w, V, F, nrhs, 0, k1, st);
    if (s != FSI_OK) return s;
    k = k1;
    std::vector<double> est(ncand, 0.0), hnum(size_t(kCandBatch) * nrhs), hden(size_t(kCandBatch) * nrhs);
    int nhist = 0;
    for (;;) {
        extract_reduced_kernel<<<cdiv(int64_t(k) * std::max(k, nrhs), 256), 256, 0, st>>>(w.P, w.ldp, w.Pf, k, nrhs, KR,
                                                                                        DR, MR, fR);
        GR_CUDA(cudaGetLastError());
        for (int f0 = 0; f0 < ncand; f0 += kCandBatch) {
            const int Fb = std::min(kCandBatch, ncand - f0);
            ReducedBatch rb;
            s = reduced_solve_batch(k, KR, DR, MR, fR, nrhs, cand + f0, Fb, w.rws, w.rws_bytes, rb, st);
            if (s != FSI_OK) return s;
            proxy_kernel<<<dim3(nrhs, Fb), 256, size_t(3) * k * sizeof(double2), st>>>(
                rb.G, rb.cs, rb.omega, k, nrhs, w.Gf, w.Gs, w.ldg, w.Hf, w.Hs, w.ldg, w.fnf, w.fns, w.num, w.den);
            GR_CUDA(cudaGetLastError());
            GR_CUDA(cudaMemcpyAsync(hnum.data(), w.num, sizeof(double) * Fb * nrhs, cudaMemcpyDeviceToHost, st));
            GR_CUDA(cudaMemcpyAsync(hden.data(), w.den, sizeof(double) * Fb * nrhs, cudaMemcpyDeviceToHost, st));
            GR_CUDA(cudaStreamSynchronize(st));
            for (int i = 0; i < Fb; ++i) {
                double a = 0.0, b = 0.0;
                for (int cc = 0; cc < nrhs; ++cc) {
                    a += std::max(0.0, hnum[size_t(i) * nrhs + cc]);
                    b += hden[size_t(i) * nrhs + cc];
                }
                est[f0 + i] = b > 0.0 ? std::sqrt(a / b) : 0.0;
            }
        }
        const double emax = *std::max_element(est.begin(), est.end());
        if (hist_out && nhist < o.max_shifts) hist_out[nhist] = emax;
        ++nhist;
        if (emax <= o.tol || int(shifts.size()) >= o.max_shifts || k >= o.kmax) break;
        auto allowed = [&](int i) {
            for (double sh : shifts)
                if (!(std::fabs(cand[i] - sh) > step * 1.0001)) return false;
            return true;
        };
        auto pick = [&](const std::vector<double>& score) {
            std::vector<int> order(ncand);
            std::iota(order.begin(), order.end(), 0);
            std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return score[a] > score[b]; });
            for (int i : order)
                if (allowed(i)) return i;
            return -1;
        };
        int inext = -1;
        if (o.mlp) {
            // learned estimate of the output error; the residual estimate confirms the choice
            std::vector<float> hx(size_t(ncand) * 5), hy(ncand);
            features(cand, ncand, shifts.data(), int(shifts.size()), est.data(), cand[0], cand[ncand - 1], hx.data());
            for (int f0 = 0; f0 < ncand; f0 += kCandBatch) {
                const int Fb = std::min(kCandBatch, ncand - f0);
                GR_CUDA(cudaMemcpyAsync(w.xf, hx.data() + size_t(f0) * 5, sizeof(float) * Fb * 5,
                                        cudaMemcpyHostToDevice, st));
                s = mlp_predict(o.mlp, w.xf, Fb, w.yf, st);
                if (s != FSI_OK) return s;
                GR_CUDA(cudaMemcpyAsync(hy.data() + f0, w.yf, sizeof(float) * Fb, cudaMemcpyDeviceToHost, st));
                GR_CUDA(cudaStreamSynchronize(st));
            }
            const int i = pick(std::vector<double>(hy.begin(), hy.end()));
            if (i >= 0 && est[i] > o.tol) inext = i;
        }
        if (inext < 0) inext = pick(est);
        if (inext < 0) break;
        double nxt = cand[inext];
        shifts.push_back(nxt);
        s = rom_build_append<R>(d, d_model, &nxt, 1, o.q, F, nrhs, o.kmax, o.build, w.build, w.build_bytes, V, k, &k1,
                                st, store);
        if (s != FSI_OK) return s;
        s = grow_gram(m, w, V, F, nrhs, k, k1, st);
        if (s != FSI_OK) return s;
        k = k1;
    }
    if (rcv && CR && nrcv > 0) {
        gather_rows_kernel<<<cdiv(int64_t(k) * nrcv, 256), 256, 0, st>>>(V, d.n, k, rcv, nrcv, CR);
        GR_CUDA(cudaGetLastError());
    }
    GR_CUDA(cudaStreamSynchronize(st));
    *k_out = k;
    for (size_t i = 0; i < shifts.size(); ++i) shifts_out[i] = shifts[i];
    *nshift_out = int(shifts.size());
    if (est_out) std::copy(est.begin(), est.end(), est_out);
    return FSI_OK;
}

// err[f] = |p_ref[f] - p[f]|_F / |p_ref[f]|_F over the m = nrcv * nrhs outputs of frequency f
__global__ void output_error_kernel(const double2* pref, const double2* p, int nf, int m, double* err) {
    const int f = blockIdx.x;
    if (f >= nf) return;
    double a = 0.0, b = 0.0;
    for (int q = threadIdx.x; q < m; q += blockDim.x) {
        const double2 r = pref[int64_t(f) * m + q], x = p[int64_t(f) * m + q];
        const double dx = x.x - r.x, dy = x.y - r.y;
        a += dx * dx + dy * dy;
        b += r.x * r.x + r.y * r.y;
    }
    __shared__ double sa[32], sb[32];
    for (int off = 16; off > 0; off >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, off);
        b += __shfl_down_sync(0xffffffffu, b, off);
    }
    if ((threadIdx.x & 31) == 0) {
        sa[threadIdx.x >> 5] = a;
        sb[threadIdx.x >> 5] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double ta = 0.0, tb = 0.0;
        for (int w = 0; w < int(blockDim.x >> 5); ++w) {
            ta += sa[w];
            tb += sb[w];
        }
        err[f] = tb > 0.0 ? sqrt(ta / tb) : 0.0;
    }
}

struct WindowResult {
    double lo, hi, maxest;
    int k, nshift, nreused;
};

// columns of the moment store of one rom_windows call: the Krylov blocks of up to four
// nested windows' expansion points (deeper ancestors' points are recomputed when needed)
inline int64_t store_cols(const fsi_greedy_opts& g, int nrhs) { return int64_t(4) * g.max_shifts * g.q * nrhs; }

// l-fROM windows: greedy ROM per window of candidates; a window whose greedy stops above tol
// (point or column budget spent) is bisected, down to min_points candidates, at most
// max_windows windows in all.  Window w's reduced matrices go to slot w of the outputs.
// Cross-window reuse (o.reuse): a window starts from the expansion points of the windows it
// was split from that lie in its band, instead of fresh quarter-midpoint points; their
// Krylov blocks are copied from the moment store (no factorisation or moment solve) and
// CGS2-appended, and only points whose blocks were not kept are recomputed.  Windows are
// processed depth first, so the store holds the blocks of the current window's ancestors
// (and of its finished siblings' subtrees, dropped before the next window starts).
template <typename R>
fsi_status run_windows(const fsi_dims& d, const void* d_model, const double2* F, int nrhs, const double* cand,
                       int ncand, const fsi_window_opts& o, void* ws, size_t ws_bytes, double2* V, const int32_t* rcv,
                       int nrcv, double2* KR, double2* DR, double2* MR, double2* fR, double2* CR,
                       MomentStore* store, void* aws, size_t aws_bytes, std::vector<WindowResult>& out,
                       cudaStream_t st) {
    const int K = o.greedy.kmax;
    struct Range {
        int i0, i1;
    };
    struct Ancestor {
        int i0, i1;
        std::vector<double> shifts;
    };
    // initial partition: init_windows windows of (nearly) equal candidate counts
    std::vector<Range> todo;
    {
        const int nw0 = std::max(1, std::min(o.init_windows, std::max(1, ncand / std::max(1, o.min_points))));
        for (int i = 0; i < nw0; ++i) todo.push_back(Range{int(int64_t(ncand) * i / nw0), int(int64_t(ncand) * (i + 1) / nw0)});
    }
    std::vector<Ancestor> anc;   // bisected windows, outermost first
    std::vector<double> shifts(o.greedy.max_shifts), hist(o.greedy.max_shifts), est(ncand);
    out.clear();
    while (!todo.empty()) {
        const Range r = todo.front();
        todo.erase(todo.begin());
        const int nc = r.i1 - r.i0;
        const double* c = cand + r.i0;
        auto contains = [&](int lo, int hi) { return lo <= r.i0 && r.i1 <= hi; };
        while (!anc.empty() && !contains(anc.back().i0, anc.back().i1)) anc.pop_back();
        std::vector<double> seed, init;
        int k = 0;
        if (o.reuse && store) {
            // finished subtrees' blocks sit on top of the store: drop them
            while (!store->blocks.empty() && !contains(store->blocks.back().lo, store->blocks.back().hi))
                store->blocks.pop_back();
            store->used = store->blocks.empty() ? 0 : store->blocks.back().col0 + store->blocks.back().ncol;
            store->lo = r.i0;
            store->hi = r.i1;
            std::vector<double> inband;   // ancestors' points in this band, first occurrence order
            for (const Ancestor& a : anc)
                for (double sh : a.shifts)
                    if (sh >= c[0] && sh <= c[nc - 1] && std::find(inband.begin(), inband.end(), sh) == inband.end())
                        inband.push_back(sh);
            if (int(inband.size()) > o.greedy.max_shifts) inband.resize(o.greedy.max_shifts);
            for (double sh : inband) {
                const MomentBlock* blk = nullptr;
                for (const MomentBlock& b : store->blocks)
                    if (b.shift == sh) blk = &b;
                if (blk) {
                    fsi_status s = rom_append_columns(V, d.n, k, K, store->buf + blk->col0 * d.n, blk->ncol, aws,
                                                      aws_bytes, st);
                    if (s != FSI_OK) return s;
                    seed.push_back(sh);
                } else {
                    init.push_back(sh);
                }
            }
        }
        if (seed.empty() && init.empty()) {
            // initial points: the candidates nearest the midpoints of init_points equal parts of
            // the window (4 parts: the quarter midpoints)
            const int npts = o.init_points > 0 ? o.init_points : 4;
            for (int qq = 0; qq < npts && int(init.size()) < o.greedy.max_shifts; ++qq) {
                const double t = c[0] + (c[nc - 1] - c[0]) * (qq + 0.5) / double(npts);
                int best = 0;
                for (int i = 1; i < nc; ++i)
                    if (std::fabs(c[i] - t) < std::fabs(c[best] - t)) best = i;
                if (std::find(init.begin(), init.end(), c[best]) == init.end()) init.push_back(c[best]);
            }
        }
        const size_t slot = out.size();
        int kw = 0, nsh = 0;
        fsi_status s = run_greedy<R>(d, d_model, F, nrhs, c, nc, init.data(), int(init.size()), o.greedy, ws, ws_bytes,
                                     V, &kw, KR + slot * K * K, DR + slot * K * K, MR + slot * K * K,
                                     fR + slot * K * nrhs, rcv, nrcv, CR ? CR + slot * nrcv * K : nullptr,
                                     shifts.data(), &nsh, est.data(), hist.data(), st, k, seed.data(),
                                     int(seed.size()), o.reuse ? store : nullptr);
        if (s != FSI_OK) return s;
        const double mx = *std::max_element(est.begin(), est.begin() + nc);
        const bool can_split = nc >= 2 * std::max(1, o.min_points) &&
                               int(out.size() + todo.size()) + 2 <= o.max_windows;
        if (mx > o.greedy.tol && can_split) {
            const int mid = r.i0 + nc / 2;
            todo.insert(todo.begin(), Range{mid, r.i1});
            todo.insert(todo.begin(), Range{r.i0, mid});
            anc.push_back(Ancestor{r.i0, r.i1, std::vector<double>(shifts.begin(), shifts.begin() + nsh)});
            continue;
        }
        out.push_back(WindowResult{c[0], c[nc - 1], mx, kw, nsh, int(seed.size())});
    }
    return FSI_OK;
}

size_t greedy_ws_bytes(const fsi_dims& d, int nrhs, const fsi_greedy_opts& o) {
    Carver c(nullptr, 0);
    GreedyWS w;
    if (o.build.precision == FSI_FP64)
        w.carve<double>(c, d, nrhs, o);
    else
        w.carve<float>(c, d, nrhs, o);
    return align_up(c.used);
}

}  // namespace

}  // namespace fsi

using namespace fsi;

extern "C" {

fsi_status rom_output_error(const fsi_c64* p_ref, const fsi_c64* p, int nf, int nout, double* err, void* stream) {
    if (!(p_ref && p && err && nf > 0 && nout > 0)) {
        set_error("rom_output_error: bad arguments");
        return FSI_EINVAL;
    }
    output_error_kernel<<<nf, 128, 0, static_cast<cudaStream_t>(stream)>>>(
        reinterpret_cast<const double2*>(p_ref), reinterpret_cast<const double2*>(p), nf, nout, err);
    GR_CUDA(cudaGetLastError());
    return FSI_OK;
}

fsi_status rom_features(const double* cand_hz, int ncand, const double* shifts_hz, int nshift, const double* est,
                        double lo, double hi, float* X_out) {
    if (!(cand_hz && est && X_out && ncand > 0 && nshift >= 0 && (nshift == 0 || shifts_hz))) {
        set_error("rom_features: bad arguments");
        return FSI_EINVAL;
    }
    features(cand_hz, ncand, shifts_hz, nshift, est, lo, hi, X_out);
    return FSI_OK;
}

fsi_status rom_greedy_workspace(const fsi_dims* dims, int nrhs, const fsi_greedy_opts* o, size_t* bytes) {
    if (!(dims && o && bytes && nrhs > 0 && nrhs <= 8 && o->q > 0 && o->kmax > 0)) {
        set_error("rom_greedy_workspace: bad arguments");
        return FSI_EINVAL;
    }
    *bytes = greedy_ws_bytes(*dims, nrhs, *o);
    return FSI_OK;
}

fsi_status rom_windows_workspace(const fsi_dims* dims, int nrhs, const fsi_window_opts* o, size_t* bytes) {
    if (!(dims && o && bytes && nrhs > 0 && nrhs <= 8 && o->greedy.q > 0 && o->greedy.kmax > 0)) {
        set_error("rom_windows_workspace: bad arguments");
        return FSI_EINVAL;
    }
    Carver c(nullptr, 0);
    c.take<char>(greedy_ws_bytes(*dims, nrhs, o->greedy));
    c.take<double2>(size_t(dims->n) * o->greedy.kmax);   // basis scratch
    if (o->reuse) {
        c.take<char>(rom_append_ws(dims->n, o->greedy.kmax));
        c.take<double2>(size_t(dims->n) * store_cols(o->greedy, nrhs));
    }
    *bytes = align_up(c.used);
    return FSI_OK;
}

fsi_status rom_windows(const fsi_dims* dims, const void* d_model, const fsi_c64* F, int nrhs, const double* cand_hz,
                       int ncand, const fsi_window_opts* o, void* ws, size_t ws_bytes, const int32_t* rcv, int nrcv,
                       fsi_c64* KR, fsi_c64* DR, fsi_c64* MR, fsi_c64* fR, fsi_c64* CR, int* nwin_out,
                       double* lo_out, double* hi_out, int* k_out, int* nshift_out, double* maxest_out,
                       int* nreused_out, void* stream) {
    if (!(dims && d_model && F && cand_hz && o && ws && rcv && KR && DR && MR && fR && CR && nwin_out && lo_out &&
          hi_out && k_out && nshift_out && maxest_out)) {
        set_error("rom_windows: NULL argument");
        return FSI_EINVAL;
    }
    const fsi_greedy_opts& g = o->greedy;
    if (!(nrhs > 0 && nrhs <= 8 && nrcv > 0 && ncand > 0 && g.q > 0 && g.kmax > 0 && g.kmax <= dims->n &&
          g.kmax <= 1024 && g.max_shifts >= 1 && o->max_windows >= 1 && o->min_points >= 1)) {
        set_error("rom_windows: bad sizes");
        return FSI_EINVAL;
    }
    if (!(g.build.precision == FSI_FP64 || g.build.precision == FSI_FP32_IR || g.build.precision == FSI_BF16X6_IR)) {
        set_error("rom_windows: unknown precision");
        return FSI_EINVAL;
    }
    for (int i = 0; i < ncand; ++i)
        if (!(cand_hz[i] > 0.0) || (i > 0 && !(cand_hz[i] > cand_hz[i - 1]))) {
            set_error("rom_windows: candidates must be positive and increasing");
            return FSI_EINVAL;
        }
    Carver c(ws, ws_bytes);
    const size_t gbytes = greedy_ws_bytes(*dims, nrhs, g);
    void* gws = c.take<char>(gbytes);
    double2* V = c.take<double2>(size_t(dims->n) * g.kmax);
    MomentStore store;
    void* aws = nullptr;
    size_t abytes = 0;
    if (o->reuse) {
        abytes = rom_append_ws(dims->n, g.kmax);
        aws = c.take<char>(abytes);
        store.cap = store_cols(g, nrhs);
        store.buf = c.take<double2>(size_t(dims->n) * store.cap);
    }
    if (!c.fits()) {
        set_error("rom_windows workspace too small: need " + std::to_string(align_up(c.used)) + " bytes");
        return FSI_ENOMEM;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    auto m2 = [](fsi_c64* p) { return reinterpret_cast<double2*>(p); };
    std::vector<WindowResult> out;
    const double2* Fd = reinterpret_cast<const double2*>(F);
    MomentStore* sp = o->reuse ? &store : nullptr;
    fsi_status s =
        g.build.precision == FSI_FP64
            ? run_windows<double>(*dims, d_model, Fd, nrhs, cand_hz, ncand, *o, gws, gbytes, V, rcv, nrcv, m2(KR),
                                  m2(DR), m2(MR), m2(fR), m2(CR), sp, aws, abytes, out, st)
            : run_windows<float>(*dims, d_model, Fd, nrhs, cand_hz, ncand, *o, gws, gbytes, V, rcv, nrcv, m2(KR),
                                 m2(DR), m2(MR), m2(fR), m2(CR), sp, aws, abytes, out, st);
    if (s != FSI_OK) return s;
    *nwin_out = int(out.size());
    for (size_t w = 0; w < out.size(); ++w) {
        lo_out[w] = out[w].lo;
        hi_out[w] = out[w].hi;
        k_out[w] = out[w].k;
        nshift_out[w] = out[w].nshift;
        maxest_out[w] = out[w].maxest;
        if (nreused_out) nreused_out[w] = out[w].nreused;
    }
    return FSI_OK;
}

fsi_status rom_windows_sweep_workspace(int kmax, int nrhs, int batch, size_t* bytes) {
    if (!(kmax > 0 && nrhs > 0 && batch > 0 && bytes)) {
        set_error("rom_windows_sweep_workspace: bad arguments");
        return FSI_EINVAL;
    }
    *bytes = reduced_solve_ws(kmax, nrhs, batch);
    return FSI_OK;
}

fsi_status rom_windows_sweep(int nwin, const double* lo, const double* hi, const int* k, int kmax,
                             const fsi_c64* KR, const fsi_c64* DR, const fsi_c64* MR, const fsi_c64* fR,
                             const fsi_c64* CR, int nrhs, int nrcv, const double* f_hz, int nf, int batch, void* ws,
                             size_t ws_bytes, fsi_c64* p_out, double* spl_out, void* stream) {
    if (!(nwin > 0 && lo && hi && k && KR && DR && MR && fR && CR && f_hz && ws && p_out && kmax > 0 && nrhs > 0 &&
          nrcv > 0 && nf > 0 && batch > 0)) {
        set_error("rom_windows_sweep: bad arguments");
        return FSI_EINVAL;
    }
    for (int i = 1; i < nf; ++i)
        if (!(f_hz[i] > f_hz[i - 1])) {
            set_error("rom_windows_sweep: frequencies must be increasing");
            return FSI_EINVAL;
        }
    for (int w = 0; w < nwin; ++w)
        if (!(k[w] > 0 && k[w] <= kmax && lo[w] <= hi[w] && (w == 0 || lo[w] > hi[w - 1]))) {
            set_error("rom_windows_sweep: windows must be ordered and non-overlapping with 0 < k <= kmax");
            return FSI_EINVAL;
        }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // each frequency goes to the window containing it, else to the nearer neighbour
    std::vector<int> owner(nf);
    for (int i = 0, w = 0; i < nf; ++i) {
        while (w + 1 < nwin && f_hz[i] > hi[w] && (f_hz[i] >= lo[w + 1] || f_hz[i] - hi[w] > lo[w + 1] - f_hz[i])) ++w;
        owner[i] = w;
    }
    const double2* KRd = reinterpret_cast<const double2*>(KR);
    const double2* DRd = reinterpret_cast<const double2*>(DR);
    const double2* MRd = reinterpret_cast<const double2*>(MR);
    const double2* fRd = reinterpret_cast<const double2*>(fR);
    const double2* CRd = reinterpret_cast<const double2*>(CR);
    double2* pd = reinterpret_cast<double2*>(p_out);
    for (int i0 = 0; i0 < nf;) {
        const int w = owner[i0];
        int i1 = i0;
        while (i1 < nf && owner[i1] == w && i1 - i0 < batch) ++i1;
        const size_t slot = size_t(w);
        ReducedBatch rb;
        fsi_status s = reduced_solve_batch(k[w], KRd + slot * kmax * kmax, DRd + slot * kmax * kmax,
                                           MRd + slot * kmax * kmax, fRd + slot * kmax * nrhs, nrhs, f_hz + i0,
                                           i1 - i0, ws, ws_bytes, rb, st);
        if (s != FSI_OK) return s;
        s = reduced_receivers(rb, CRd + slot * nrcv * kmax, nrcv, pd + int64_t(i0) * nrcv * nrhs,
                              spl_out ? spl_out + int64_t(i0) * nrcv * nrhs : nullptr, st);
        if (s != FSI_OK) return s;
        i0 = i1;
    }
    GR_CUDA(cudaStreamSynchronize(st));
    return FSI_OK;
}

fsi_status rom_greedy(const fsi_dims* dims, const void* d_model, const fsi_c64* F, int nrhs, const double* cand_hz,
                      int ncand, const double* init_hz, int ninit, const fsi_greedy_opts* o, void* ws,
                      size_t ws_bytes, fsi_c64* V, int* k_out, fsi_c64* KR, fsi_c64* DR, fsi_c64* MR, fsi_c64* fR,
                      const int32_t* rcv, int nrcv, fsi_c64* CR, double* shifts_out, int* nshift_out,
                      double* est_out, double* hist_out, void* stream) {
    if (!(dims && d_model && F && cand_hz && o && ws && V && k_out && KR && DR && MR && fR && shifts_out &&
          nshift_out)) {
        set_error("rom_greedy: NULL argument");
        return FSI_EINVAL;
    }
    if (!(nrhs > 0 && nrhs <= 8 && ncand > 0 && ninit >= 0 && (ninit == 0 || init_hz) && o->q > 0 && o->kmax > 0 &&
          o->kmax <= dims->n && o->kmax <= 1024 && o->max_shifts > 0 && o->max_shifts >= ninit)) {
        set_error("rom_greedy: bad sizes");
        return FSI_EINVAL;
    }
    if (!(o->build.precision == FSI_FP64 || o->build.precision == FSI_FP32_IR || o->build.precision == FSI_BF16X6_IR)) {
        set_error("rom_greedy: unknown precision");
        return FSI_EINVAL;
    }
    for (int i = 0; i < ncand; ++i)
        if (!(cand_hz[i] > 0.0) || (i > 0 && !(cand_hz[i] > cand_hz[i - 1]))) {
            set_error("rom_greedy: candidates must be positive and increasing");
            return FSI_EINVAL;
        }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    auto d2 = [](const fsi_c64* p) { return reinterpret_cast<const double2*>(p); };
    auto m2 = [](fsi_c64* p) { return reinterpret_cast<double2*>(p); };
    if (o->build.precision == FSI_FP64)
        return run_greedy<double>(*dims, d_model, d2(F), nrhs, cand_hz, ncand, init_hz, ninit, *o, ws, ws_bytes, m2(V),
                                  k_out, m2(KR), m2(DR), m2(MR), m2(fR), rcv, nrcv, CR ? m2(CR) : nullptr, shifts_out,
                                  nshift_out, est_out, hist_out, st);
    return run_greedy<float>(*dims, d_model, d2(F), nrhs, cand_hz, ncand, init_hz, ninit, *o, ws, ws_bytes, m2(V),
                             k_out, m2(KR), m2(DR), m2(MR), m2(fR), rcv, nrcv, CR ? m2(CR) : nullptr, shifts_out,
                             nshift_out, est_out, hist_out, st);
}

}  // extern "C"
