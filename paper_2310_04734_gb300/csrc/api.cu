// C ABI entry points and host-side orchestration of the full-order sweep.
//
// Full-order sweep (paper Sec. 2, Eq. 1; Sec. 3.3, Eq. 8).  For a batch of
// frequencies the scaled slab-ordered matrix is factored window by window:
// the window of step k stacks the current rows of slab k (block columns
// k, k+1, k+2) on the rows of slab k+1; its first b columns are eliminated
// with partial pivoting over all 2b rows (a band LU: rows of slab k+1 may
// pivot for slab k), the pivot rows are kept for the backward sweep, the
// multipliers of slab k+1 for the forward sweep, and the Schur tail becomes
// the current rows of slab k+1.  Solves run slab by slab forward and back.
// FP32 factors are refined against the FP64 residual until the relative
// residual of the scaled system reaches the tolerance.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <sstream>
#include <string>
#include <vector>

#include "fsi_internal.h"
#include "kernels.cuh"
#include "engine.h"
#include "prof.h"

namespace fsi {

namespace {
thread_local std::string g_last_error;
}

void set_error(const std::string& msg) { g_last_error = msg; }

#define FSI_CUDA(call)                                                                                 \
    do {                                                                                               \
        cudaError_t e_ = (call);                                                                       \
        if (e_ != cudaSuccess) {                                                                       \
            std::ostringstream o_;                                                                     \
            o_ << #call << ": " << cudaGetErrorString(e_) << " (" << __FILE__ << ":" << __LINE__ << ")"; \
            set_error(o_.str());                                                                       \
            return FSI_ECUDA;                                                                          \
        }                                                                                              \
    } while (0)

#define FSI_CHECK_LAUNCH() FSI_CUDA(cudaGetLastError())

#define FSI_REQUIRE(cond, msg)      \
    do {                            \
        if (!(cond)) {              \
            set_error(msg);         \
            return FSI_EINVAL;      \
        }                           \
    } while (0)

DevModel dev_model(const fsi_dims& d, const void* blob) {
    const ModelLayout L = model_layout(d);
    const char* b = static_cast<const char*>(blob);
    DevModel m;
    m.rowptr = reinterpret_cast<const int32_t*>(b + L.rowptr);
    m.col = reinterpret_cast<const int32_t*>(b + L.col);
    m.K = reinterpret_cast<const double2*>(b + L.K);
    m.M = reinterpret_cast<const double*>(b + L.M);
    m.D = reinterpret_cast<const double2*>(b + L.D);
    m.kdiag = reinterpret_cast<const double*>(b + L.kdiag);
    m.cbase = reinterpret_cast<const double*>(b + L.cbase);
    m.rbase = reinterpret_cast<const double*>(b + L.rbase);
    m.n = d.n;
    m.b = d.b;
    m.nz = d.nz;
    m.npl = d.n_press_slab;
    m.rho = d.rho;
    return m;
}

template <typename R>
fsi_status factor_batch(const DevModel& m, Factor<R>& fc, int F, const double* d_omega, cudaStream_t st) {
    const int b = m.b, nz = m.nz, ld = 3 * b;
    FSI_CUDA(cudaMemsetAsync(fc.status, 0, sizeof(int32_t) * F, st));
    FSI_CUDA(cudaMemsetAsync(fc.tc.err, 0, sizeof(int32_t), st));
    launch_form_rows<R>(m, fc.G, fc.sG, ld, F, d_omega, 0, 0, 0, ld, st);
    FSI_CHECK_LAUNCH();
    for (int k = 0; k < nz; ++k) {
        const int m_rows = (k + 1 < nz) ? 2 * b : b;
        const int ncols = std::min(3, nz - k) * b;
        if (k + 1 < nz) launch_form_rows<R>(m, fc.G, fc.sG, ld, F, d_omega, k + 1, b, k, ld, st);
        partial_lu<R>(fc.G, fc.sG, ld, F, m_rows, ncols, b, fc.ipiv + int64_t(k) * b, fc.sP, fc.status, st,
                      fc.use_tc ? &fc.tc : nullptr);
        launch_slab_shift<R>(fc.G, fc.sG, F, b, m_rows, fc.U + int64_t(k) * b * 3 * b, fc.sU,
                             fc.L + int64_t(k) * b * b, fc.sL, fc.ipiv + int64_t(k) * b, fc.sP,
                             fc.perm + int64_t(k) * 2 * b, fc.sPerm, st);
        FSI_CHECK_LAUNCH();
    }
    return FSI_OK;
}

template <typename R>
fsi_status solve_batch(const DevModel& m, Factor<R>& fc, int F, typename Cplx<R>::T* y, int64_t sY, int nrhs,
                       cudaStream_t st, const int32_t* flist, int nF) {
    const int b = m.b, nz = m.nz;
    const int Fl = flist ? nF : F;
    if (Fl <= 0) return FSI_OK;
    for (int k = 0; k < nz; ++k) {
        launch_slab_solve_fwd<R>(fc.U + int64_t(k) * b * 3 * b, fc.L + int64_t(k) * b * b, fc.sU, fc.sL,
                                 fc.perm + int64_t(k) * 2 * b, fc.sPerm, y, sY, m.n, b, k, nz, nrhs, Fl, flist, st);
    }
    for (int k = nz - 1; k >= 0; --k) {
        launch_slab_solve_bwd<R>(fc.U + int64_t(k) * b * 3 * b, fc.sU, y, sY, m.n, b, k, nz, nrhs, Fl, flist, st);
    }
    FSI_CHECK_LAUNCH();
    return FSI_OK;
}

// ------------------------------------------------------------------ sweep workspace
template <typename R>
struct SweepWS {
    using T2 = typename Cplx<R>::T;
    Factor<R> fc;
    double* omega = nullptr;
    double2* xhat = nullptr;
    double2* rhat = nullptr;
    T2* y = nullptr;
    double* norms = nullptr;
    double* fnorms = nullptr;
    double* absn = nullptr;
    double2* Fd = nullptr;
    int32_t* rcvd = nullptr;
    double2* pb = nullptr;
    double* splb = nullptr;
    void* gws = nullptr;
    size_t gws_bytes = 0;
    int64_t sV = 0;

    void carve(Carver& c, const fsi_dims& d, int F, int nrhs, int nrcv, bool host_io, int gmres_restart,
               int planes) {
        fc.carve(c, d, F, nrhs, planes);
        sV = int64_t(nrhs) * d.n;
        omega = c.take<double>(F);
        xhat = c.take<double2>(size_t(F) * sV);
        rhat = c.take<double2>(size_t(F) * sV);
        y = c.take<T2>(size_t(F) * sV);
        norms = c.take<double>(size_t(F) * nrhs);
        fnorms = c.take<double>(size_t(F) * nrhs);
        absn = c.take<double>(size_t(F) * nrhs);
        if (host_io) {
            Fd = c.take<double2>(size_t(d.n) * nrhs);
            rcvd = c.take<int32_t>(nrcv);
            pb = c.take<double2>(size_t(F) * nrcv * nrhs);
            splb = c.take<double>(size_t(F) * nrcv * nrhs);
        }
        if (gmres_restart > 0) {
            gws_bytes = gmres_ws_bytes(d.n, F * nrhs, gmres_restart);
            gws = c.take<char>(gws_bytes);
        }
    }
};

bool known_precision(int p) {
    return p == FSI_FP64 || p == FSI_FP32_IR || p == FSI_BF16X6_IR || p == FSI_BF16_IR;
}

// BF16 planes per operand of the tensor-core updates for a precision (0: none)
int tc_planes(int p) { return p == FSI_BF16X6_IR ? 3 : (p == FSI_BF16_IR ? 1 : 0); }

int gmres_restart_of(const fsi_solve_opts& o) {
    if (o.refine != FSI_REFINE_GMRES) return 0;
    return o.restart > 0 ? o.restart : 20;
}

fsi_status check_dims(const fsi_dims* d) {
    FSI_REQUIRE(d, "dims is NULL");
    FSI_REQUIRE(d->b > 0 && d->nz >= 3 && d->n == int64_t(d->b) * d->nz && d->nnz > 0, "inconsistent fsi_dims");
    return FSI_OK;
}

template <typename R>
size_t sweep_ws_bytes(const fsi_dims& d, int F, int nrhs, int nrcv, bool host_io, int restart, int planes) {
    Carver c(nullptr, 0);
    SweepWS<R> w;
    w.carve(c, d, F, nrhs, nrcv, host_io, restart, planes);
    return align_up(c.used);
}

template <typename R>
fsi_status ir_solve(const DevModel& m, Factor<R>& fc, int Fb, const double* d_omega, const double2* Bdev, int nrhs,
                    double2* xhat, double2* rhat, typename Cplx<R>::T* y, double* norms, double* fnorms,
                    double* absn, int64_t sV, int max_it, double tol, std::vector<int>& it_done,
                    std::vector<double>& rel, cudaStream_t st, int64_t sB) {
    std::vector<double> hn(size_t(Fb) * nrhs), hf(size_t(Fb) * nrhs), ha(size_t(Fb) * nrhs);
    FSI_CUDA(cudaMemsetAsync(fnorms, 0, sizeof(double) * Fb * nrhs, st));
    launch_residual(m, d_omega, 0.0, Fb, nullptr, sV, Bdev, nrhs, rhat, sV, fnorms, true, st, nullptr, sB);
    FSI_CHECK_LAUNCH();
    FSI_CUDA(cudaMemcpyAsync(norms, fnorms, sizeof(double) * Fb * nrhs, cudaMemcpyDeviceToDevice, st));
    FSI_CUDA(cudaMemcpyAsync(hf.data(), fnorms, sizeof(double) * Fb * nrhs, cudaMemcpyDeviceToHost, st));
    FSI_CUDA(cudaMemsetAsync(xhat, 0, sizeof(double2) * Fb * sV, st));
    it_done.assign(Fb, -1);
    rel.assign(Fb, 0.0);
    for (int it = 1; it <= max_it; ++it) {
        launch_to_low<R>(rhat, sV, norms, y, sV, m.n, nrhs, Fb, st);
        fsi_status s = solve_batch<R>(m, fc, Fb, y, sV, nrhs, st);
        if (s != FSI_OK) return s;
        launch_update<R>(xhat, sV, norms, y, sV, m.n, nrhs, Fb, nullptr, st);
        FSI_CUDA(cudaMemsetAsync(norms, 0, sizeof(double) * Fb * nrhs, st));
        FSI_CUDA(cudaMemsetAsync(absn, 0, sizeof(double) * Fb * nrhs, st));
        launch_residual(m, d_omega, 0.0, Fb, xhat, sV, Bdev, nrhs, rhat, sV, norms, true, st, absn, sB);
        FSI_CHECK_LAUNCH();
        FSI_CUDA(cudaMemcpyAsync(hn.data(), norms, sizeof(double) * Fb * nrhs, cudaMemcpyDeviceToHost, st));
        FSI_CUDA(cudaMemcpyAsync(ha.data(), absn, sizeof(double) * Fb * nrhs, cudaMemcpyDeviceToHost, st));
        FSI_CUDA(cudaStreamSynchronize(st));
        bool all = true;
        for (int f = 0; f < Fb; ++f) {
            double r = 0.0;
            bool conv = true;
            for (int cc = 0; cc < nrhs; ++cc) {
                const size_t q = size_t(f) * nrhs + cc;
                const double den = hf[q];
                const double v = den > 0 ? std::sqrt(hn[q] / den) : 0.0;
                r = std::max(r, std::isfinite(v) ? v : INFINITY);
                const bool at_floor = std::sqrt(hn[q]) <= kResFloor * std::sqrt(ha[q]);
                if (!(v <= tol || at_floor)) conv = false;
            }
            rel[f] = r;
            if (it_done[f] < 0 && conv) it_done[f] = it;
            if (it_done[f] < 0) all = false;
        }
        if (all) break;
    }
    return FSI_OK;
}

template <typename R>
fsi_status run_sweep(const fsi_dims& d, const void* d_model, const double* f_hz, int nf, const fsi_c64* F,
                     int nrhs, const int32_t* rcv, int nrcv, const fsi_solve_opts& o, void* ws, size_t ws_bytes,
                     fsi_c64* p_out, double* spl_out, int32_t* iters_out, double* relres_out,
                     fsi_sweep_stats* stats, cudaStream_t st) {
    const int Fb_max = std::max(1, std::min(o.batch, nf));
    const bool host_io = o.host_io != 0;
    Carver c(ws, ws_bytes);
    SweepWS<R> w;
    const int restart = gmres_restart_of(o);
    w.carve(c, d, Fb_max, nrhs, nrcv, host_io, restart, tc_planes(o.precision));
    if (!c.fits()) {
        set_error("workspace too small: need " + std::to_string(align_up(c.used)) + " bytes");
        return FSI_ENOMEM;
    }
    const DevModel m = dev_model(d, d_model);
    w.fc.use_tc = tc_planes(o.precision) > 0;
    prof().reset(o.profile != 0);
    const double2* Fdev = reinterpret_cast<const double2*>(F);
    const int32_t* rcvdev = rcv;
    if (host_io) {
        FSI_CUDA(cudaMemcpyAsync(w.Fd, F, sizeof(double2) * d.n * nrhs, cudaMemcpyHostToDevice, st));
        FSI_CUDA(cudaMemcpyAsync(w.rcvd, rcv, sizeof(int32_t) * nrcv, cudaMemcpyHostToDevice, st));
        Fdev = w.Fd;
        rcvdev = w.rcvd;
    }
    const int max_it = o.precision == FSI_FP64 ? std::max(1, o.max_refine) : std::max(1, o.max_refine);
    const double tol = o.tol > 0 ? o.tol : 1e-8;
    std::vector<double> om(Fb_max);
    std::vector<int32_t> hstat(Fb_max);
    fsi_sweep_stats S{};
    bool singular = false;
    std::vector<int> it_done;
    std::vector<double> rel;
    for (int f0 = 0; f0 < nf; f0 += Fb_max) {
        const int Fb = std::min(Fb_max, nf - f0);
        for (int i = 0; i < Fb; ++i) om[i] = 2.0 * M_PI * f_hz[f0 + i];
        FSI_CUDA(cudaMemcpyAsync(w.omega, om.data(), sizeof(double) * Fb, cudaMemcpyHostToDevice, st));
        fsi_status s = factor_batch<R>(m, w.fc, Fb, w.omega, st);
        if (s != FSI_OK) return s;
        if (restart > 0)
            s = fgmres_solve<R>(m, w.fc, Fb, w.omega, Fdev, nrhs, w.xhat, w.rhat, w.y, w.norms, w.fnorms, w.absn, w.sV,
                                restart, (max_it + restart - 1) / restart, tol, w.gws, w.gws_bytes, it_done, rel, st);
        else
            s = ir_solve<R>(m, w.fc, Fb, w.omega, Fdev, nrhs, w.xhat, w.rhat, w.y, w.norms, w.fnorms, w.absn, w.sV, max_it,
                            tol, it_done, rel, st);
        if (s != FSI_OK) return s;
        FSI_CUDA(cudaMemcpyAsync(hstat.data(), w.fc.status, sizeof(int32_t) * Fb, cudaMemcpyDeviceToHost, st));
        int32_t htc = 0;
        FSI_CUDA(cudaMemcpyAsync(&htc, w.fc.tc.err, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        double2* pdst = host_io ? w.pb : reinterpret_cast<double2*>(p_out) + int64_t(f0) * nrcv * nrhs;
        double* sdst = host_io ? w.splb : (spl_out ? spl_out + int64_t(f0) * nrcv * nrhs : nullptr);
        launch_receivers(m, w.omega, Fb, w.xhat, w.sV, rcvdev, nrcv, nrhs, pdst, sdst, st);
        FSI_CHECK_LAUNCH();
        if (host_io) {
            FSI_CUDA(cudaMemcpyAsync(p_out + int64_t(f0) * nrcv * nrhs, w.pb, sizeof(double2) * Fb * nrcv * nrhs,
                                     cudaMemcpyDeviceToHost, st));
            if (spl_out)
                FSI_CUDA(cudaMemcpyAsync(spl_out + int64_t(f0) * nrcv * nrhs, w.splb,
                                         sizeof(double) * Fb * nrcv * nrhs, cudaMemcpyDeviceToHost, st));
        }
        FSI_CUDA(cudaStreamSynchronize(st));
        prof().collect();
        if (htc) {
            set_error("a tensor-core update gave up waiting for its loads or MMAs");
            return FSI_ETIMEOUT;
        }
        for (int f = 0; f < Fb; ++f) {
            const int its = it_done[f] < 0 ? max_it : it_done[f];
            if (iters_out) iters_out[f0 + f] = its;
            if (relres_out) relres_out[f0 + f] = rel[f];
            S.max_iters = std::max(S.max_iters, its);
            S.max_relres = std::max(S.max_relres, rel[f]);
            if (it_done[f] < 0) S.n_unconverged++;
            if (hstat[f]) singular = true;
        }
        S.n_done = f0 + Fb;
    }
    S.launches = prof().launches;
    static_assert(int(PK_COUNT) == int(FSI_K_COUNT) && int(FSI_K_COUNT) <= int(FSI_K_SLOTS) &&
                      int(PK_GEMV) == int(FSI_K_GEMV) && int(PK_SOLVE) == int(FSI_K_SOLVE) &&
                      int(PK_PACK) == int(FSI_K_PACK) && int(PK_TCGEMM) == int(FSI_K_TCGEMM),
                  "kernel classes of the profiler and the C ABI differ");
    for (int i = 0; i < PK_COUNT; ++i) {
        S.kernel_ms[i] = prof().ms[i];
        S.kernel_flops[i] = prof().flops[i];
        S.kernel_launches[i] = prof().count[i];
    }
    prof().reset(false);
    if (stats) *stats = S;
    if (singular) {
        set_error("zero or non-finite pivot in the factorisation");
        return FSI_ESINGULAR;
    }
    if (S.n_unconverged > 0 && o.precision != FSI_FP64) {
        set_error(std::to_string(S.n_unconverged) + " frequencies above tol after max_refine iterations");
        return FSI_ENOCONV;
    }
    return FSI_OK;
}

template fsi_status solve_batch<float>(const DevModel&, Factor<float>&, int, float2*, int64_t, int, cudaStream_t,
                                       const int32_t*, int);
template fsi_status solve_batch<double>(const DevModel&, Factor<double>&, int, double2*, int64_t, int, cudaStream_t,
                                        const int32_t*, int);
template fsi_status factor_batch<float>(const DevModel&, Factor<float>&, int, const double*, cudaStream_t);
template fsi_status factor_batch<double>(const DevModel&, Factor<double>&, int, const double*, cudaStream_t);
template fsi_status ir_solve<float>(const DevModel&, Factor<float>&, int, const double*, const double2*, int,
                                    double2*, double2*, float2*, double*, double*, double*, int64_t, int, double,
                                    std::vector<int>&, std::vector<double>&, cudaStream_t, int64_t);
template fsi_status ir_solve<double>(const DevModel&, Factor<double>&, int, const double*, const double2*, int,
                                     double2*, double2*, double2*, double*, double*, double*, int64_t, int, double,
                                     std::vector<int>&, std::vector<double>&, cudaStream_t, int64_t);

}  // namespace fsi

using namespace fsi;

extern "C" {

const char* fsi_status_str(fsi_status s) {
    switch (s) {
        case FSI_OK: return "ok";
        case FSI_EINVAL: return "invalid argument";
        case FSI_ENOMEM: return "buffer too small";
        case FSI_ECUDA: return "CUDA error";
        case FSI_ESINGULAR: return "singular factor";
        case FSI_ENOCONV: return "refinement did not converge";
        case FSI_ETIMEOUT: return "device wait timed out";
        case FSI_ESTATE: return "call out of order";
    }
    return "unknown status";
}

const char* fsi_last_error(void) { return g_last_error.c_str(); }

fsi_status fsi_model_dims(const fsi_model_desc* desc, fsi_dims* out) {
    FSI_REQUIRE(desc && out, "NULL argument");
    HostModel hm;
    fsi_status s = assemble_host(*desc, hm);
    if (s != FSI_OK) return s;
    *out = hm.dims;
    return FSI_OK;
}

fsi_status fsi_assemble_host(const fsi_model_desc* desc, int32_t* rowptr, int32_t* col, fsi_c64* K, double* M,
                             fsi_c64* D) {
    FSI_REQUIRE(desc && rowptr && col && K && M && D, "NULL argument");
    HostModel hm;
    fsi_status s = assemble_host(*desc, hm);
    if (s != FSI_OK) return s;
    std::memcpy(rowptr, hm.rowptr.data(), sizeof(int32_t) * hm.rowptr.size());
    std::memcpy(col, hm.col.data(), sizeof(int32_t) * hm.col.size());
    std::memcpy(K, hm.K.data(), sizeof(fsi_c64) * hm.K.size());
    std::memcpy(M, hm.M.data(), sizeof(double) * hm.M.size());
    std::memcpy(D, hm.D.data(), sizeof(fsi_c64) * hm.D.size());
    return FSI_OK;
}

fsi_status fsi_assemble(const fsi_model_desc* desc, void* d_model, size_t model_bytes, void* stream) {
    FSI_REQUIRE(desc && d_model, "NULL argument");
    FSI_REQUIRE((reinterpret_cast<uintptr_t>(d_model) % kAlign) == 0, "model buffer must be 256-byte aligned");
    HostModel hm;
    fsi_status s = assemble_host(*desc, hm);
    if (s != FSI_OK) return s;
    const ModelLayout L = model_layout(hm.dims);
    if (model_bytes < L.total) {
        set_error("model buffer too small: need " + std::to_string(L.total) + " bytes");
        return FSI_ENOMEM;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    char* b = static_cast<char*>(d_model);
    FSI_CUDA(cudaMemcpyAsync(b + L.rowptr, hm.rowptr.data(), sizeof(int32_t) * hm.rowptr.size(),
                             cudaMemcpyHostToDevice, st));
    FSI_CUDA(cudaMemcpyAsync(b + L.col, hm.col.data(), sizeof(int32_t) * hm.col.size(), cudaMemcpyHostToDevice, st));
    FSI_CUDA(cudaMemcpyAsync(b + L.K, hm.K.data(), sizeof(fsi_c64) * hm.K.size(), cudaMemcpyHostToDevice, st));
    FSI_CUDA(cudaMemcpyAsync(b + L.M, hm.M.data(), sizeof(double) * hm.M.size(), cudaMemcpyHostToDevice, st));
    FSI_CUDA(cudaMemcpyAsync(b + L.D, hm.D.data(), sizeof(fsi_c64) * hm.D.size(), cudaMemcpyHostToDevice, st));
    FSI_CUDA(cudaMemcpyAsync(b + L.kdiag, hm.kdiag.data(), sizeof(double) * hm.kdiag.size(), cudaMemcpyHostToDevice,
                             st));
    // frequency-independent factors of the equilibration: column scale = cbase (shell) or
    // |cbase| w (fluid, stored negative), row scale = rbase (shell) or |rbase| / w (fluid)
    std::vector<double> cb(hm.kdiag.size()), rb(hm.kdiag.size());
    for (size_t g = 0; g < cb.size(); ++g) {
        const double kd = hm.kdiag[g];
        const bool fluid = int64_t(g % size_t(hm.dims.b)) < hm.dims.n_press_slab;
        cb[g] = fluid ? -std::sqrt(hm.dims.rho / kd) : 1.0 / std::sqrt(kd);
        rb[g] = fluid ? -(1.0 / std::sqrt(hm.dims.rho * kd)) : 1.0 / std::sqrt(kd);
    }
    FSI_CUDA(cudaMemcpyAsync(b + L.cbase, cb.data(), sizeof(double) * cb.size(), cudaMemcpyHostToDevice, st));
    FSI_CUDA(cudaMemcpyAsync(b + L.rbase, rb.data(), sizeof(double) * rb.size(), cudaMemcpyHostToDevice, st));
    FSI_CUDA(cudaStreamSynchronize(st));
    return FSI_OK;
}

fsi_status frf_sweep_workspace(const fsi_dims* dims, const fsi_solve_opts* opts, int nrhs, int nrcv, size_t* bytes) {
    fsi_status s = check_dims(dims);
    if (s != FSI_OK) return s;
    FSI_REQUIRE(opts && bytes && nrhs > 0 && nrcv > 0 && opts->batch > 0, "bad sweep workspace arguments");
    const bool hio = opts->host_io != 0;
    const int rs = gmres_restart_of(*opts);
    FSI_REQUIRE(known_precision(opts->precision), "unknown precision");
    *bytes = opts->precision == FSI_FP64 ? sweep_ws_bytes<double>(*dims, opts->batch, nrhs, nrcv, hio, rs, 0)
                                         : sweep_ws_bytes<float>(*dims, opts->batch, nrhs, nrcv, hio, rs,
                                                                 tc_planes(opts->precision));
    return FSI_OK;
}

fsi_status frf_sweep_full(const fsi_dims* dims, const void* d_model, const double* f_hz, int nf, const fsi_c64* F,
                          int nrhs, const int32_t* rcv, int nrcv, const fsi_solve_opts* opts, void* ws,
                          size_t ws_bytes, fsi_c64* p_out, double* spl_out, int32_t* iters_out, double* relres_out,
                          fsi_sweep_stats* stats, void* stream) {
    fsi_status s = check_dims(dims);
    if (s != FSI_OK) return s;
    FSI_REQUIRE(d_model && f_hz && F && rcv && opts && ws && p_out, "NULL argument");
    FSI_REQUIRE(nf > 0 && nrhs > 0 && nrcv > 0 && opts->batch > 0, "nf, nrhs, nrcv, batch must be positive");
    FSI_REQUIRE(known_precision(opts->precision), "unknown precision");
    for (int i = 0; i < nf; ++i) FSI_REQUIRE(f_hz[i] > 0.0 && std::isfinite(f_hz[i]), "frequencies must be > 0");
    if (opts->host_io)
        for (int i = 0; i < nrcv; ++i) FSI_REQUIRE(rcv[i] >= 0 && rcv[i] < dims->n, "receiver index out of range");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (opts->precision == FSI_FP64)
        return run_sweep<double>(*dims, d_model, f_hz, nf, F, nrhs, rcv, nrcv, *opts, ws, ws_bytes, p_out, spl_out,
                                 iters_out, relres_out, stats, st);
    return run_sweep<float>(*dims, d_model, f_hz, nf, F, nrhs, rcv, nrcv, *opts, ws, ws_bytes, p_out, spl_out,
                            iters_out, relres_out, stats, st);
}

fsi_status fsi_residual(const fsi_dims* dims, const void* d_model, const double* f_hz, int nf, const fsi_c64* X,
                        const fsi_c64* F, int nrhs, fsi_c64* R, void* stream) {
    fsi_status s = check_dims(dims);
    if (s != FSI_OK) return s;
    FSI_REQUIRE(d_model && f_hz && X && F && R && nf > 0 && nrhs > 0, "bad residual arguments");
    const DevModel m = dev_model(*dims, d_model);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int64_t sV = int64_t(nrhs) * dims->n;
    for (int f = 0; f < nf; ++f) {
        launch_residual(m, nullptr, 2.0 * M_PI * f_hz[f], 1, reinterpret_cast<const double2*>(X) + f * sV, sV,
                        reinterpret_cast<const double2*>(F), nrhs, reinterpret_cast<double2*>(R) + f * sV, sV,
                        nullptr, false, st);
        FSI_CHECK_LAUNCH();
    }
    return FSI_OK;
}

fsi_status fsi_lu_workspace(int precision, int batch, int m, int ncols, int npiv, size_t* bytes) {
    FSI_REQUIRE(batch > 0 && m > 0 && ncols > 0 && npiv > 0 && npiv <= m && npiv <= ncols && bytes,
                "bad lu workspace arguments");
    FSI_REQUIRE(known_precision(precision), "unknown precision");
    size_t b = align_up(sizeof(int32_t) * size_t(batch + 1));
    if (tc_planes(precision) > 0) b += align_up(tc_workspace_bytes(batch, m, ncols, npiv, tc_planes(precision)));
    *bytes = b;
    return FSI_OK;
}

fsi_status fsi_batched_lu(int precision, int batch, int m, int ncols, int npiv, void* A, int64_t ld, int64_t sA,
                          int32_t* ipiv, void* ws, size_t ws_bytes, int* n_singular_out, void* stream) {
    FSI_REQUIRE(A && ipiv && ws && batch > 0 && m > 0 && ncols > 0, "bad batched lu arguments");
    FSI_REQUIRE(npiv > 0 && npiv <= m && npiv <= ncols && ld >= ncols && sA >= ld * m, "bad batched lu shape");
    FSI_REQUIRE(known_precision(precision), "unknown precision");
    size_t need = 0;
    fsi_status s0 = fsi_lu_workspace(precision, batch, m, ncols, npiv, &need);
    if (s0 != FSI_OK) return s0;
    FSI_REQUIRE(ws_bytes >= need, "workspace too small");
    FSI_REQUIRE(m <= 8192, "m too large for the panel kernel");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int32_t* status = static_cast<int32_t*>(ws);
    FSI_CUDA(cudaMemsetAsync(status, 0, sizeof(int32_t) * (batch + 1), st));
    if (precision == FSI_FP64) {
        partial_lu<double>(static_cast<double2*>(A), sA, int(ld), batch, m, ncols, npiv, ipiv, npiv, status, st);
    } else {
        TcCtx tc;
        const bool tensor = tc_planes(precision) > 0;
        if (tensor) {
            const size_t off = align_up(sizeof(int32_t) * size_t(batch + 1));
            tc.planes = tc_planes(precision);
            tc.a_bytes = tc_a_region_bytes(batch, m, ncols, npiv, tc.planes);
            tc.err = status + batch;
            tc.ws = static_cast<char*>(ws) + off;
            tc.ws_bytes = ws_bytes - off;
        }
        partial_lu<float>(static_cast<float2*>(A), sA, int(ld), batch, m, ncols, npiv, ipiv, npiv, status, st,
                          tensor ? &tc : nullptr);
    }
    FSI_CHECK_LAUNCH();
    if (n_singular_out || tc_planes(precision) > 0) {
        std::vector<int32_t> h(batch + 1);
        FSI_CUDA(cudaMemcpyAsync(h.data(), status, sizeof(int32_t) * (batch + 1), cudaMemcpyDeviceToHost, st));
        FSI_CUDA(cudaStreamSynchronize(st));
        int cnt = 0;
        for (int i = 0; i < batch; ++i) cnt += h[i] != 0;
        if (n_singular_out) *n_singular_out = cnt;
        if (tc_planes(precision) > 0 && h[batch]) {
            set_error("a tensor-core update gave up waiting for its loads or MMAs");
            return FSI_ETIMEOUT;
        }
    }
    return FSI_OK;
}

fsi_status fsi_set_wait_limit(int64_t spins) {
    FSI_REQUIRE(spins >= 0, "spin limit must be >= 0");
    set_tc_spin_limit(spins > int64_t(UINT32_MAX) ? UINT32_MAX : uint32_t(spins));
    return FSI_OK;
}

}  // extern "C"
