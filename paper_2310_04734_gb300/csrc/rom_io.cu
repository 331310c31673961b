// Reduced models on disk, and the check-and-re-solve step of the reduced sweep.
//
// Offline / online split (paper Sec. 3.3): the expensive part of the method
// (factorisations at the expansion points, moments, projection) is done once;
// the reduced matrices are then reused for any number of sweeps.  rom_save
// writes a reduced model (one window, or the windows of rom_windows in their
// slot layout) with its expansion points and, optionally, its projection
// bases; rom_file_info and rom_load read it back bit for bit.
//
// File layout (little endian), version 1:
//   magic "FSIROM\0\1", then a header of int32 {version, nwin, kmax, nrhs, nrcv,
//   nshift_total} and int64 n; per window double lo, hi and int32 k, nshift;
//   the expansion points (double, window by window); per window K_R, D_R, M_R
//   (k x k), f_R (k x nrhs), C_R (nrcv x k), all column-major complex128, and
//   the basis V (n x k) when n > 0; finally a 64-bit FNV-1a checksum of every
//   byte after the magic.
//
// rom_check_resolve: the full-order FP64 residual of the lifted reduced
// solutions judges each frequency (rom_residual_check); frequencies above the
// tolerance are solved again at full order (frf_sweep_full) and their outputs
// replace the reduced ones.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "fsi_internal.h"

namespace fsi {

namespace {

constexpr char kMagic[8] = {'F', 'S', 'I', 'R', 'O', 'M', 0, 1};
constexpr int32_t kVersion = 1;

struct Fnv {
    uint64_t h = 1469598103934665603ull;
    void add(const void* p, size_t n) {
        const unsigned char* c = static_cast<const unsigned char*>(p);
        for (size_t i = 0; i < n; ++i) {
            h ^= c[i];
            h *= 1099511628211ull;
        }
    }
};

struct Writer {
    FILE* f;
    Fnv sum;
    bool ok = true;
    void put(const void* p, size_t n) {
        if (!ok || n == 0) return;
        sum.add(p, n);
        ok = std::fwrite(p, 1, n, f) == n;
    }
};

struct Reader {
    FILE* f;
    Fnv sum;
    bool ok = true;
    void get(void* p, size_t n) {
        if (!ok || n == 0) return;
        ok = std::fread(p, 1, n, f) == n;
        if (ok) sum.add(p, n);
    }
};

fsi_status fail(fsi_status s, const std::string& msg) {
    set_error(msg);
    return s;
}

// One contiguous array: host pointer as is, device pointer through a host staging copy.
fsi_status save_array(Writer& w, const void* src, size_t bytes, bool dev, std::vector<char>& stage,
                      cudaStream_t st) {
    if (bytes == 0) return FSI_OK;
    if (!dev) {
        w.put(src, bytes);
        return FSI_OK;
    }
    stage.resize(bytes);
    cudaError_t e = cudaMemcpyAsync(stage.data(), src, bytes, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail(FSI_ECUDA, std::string("rom_save: ") + cudaGetErrorString(e));
    w.put(stage.data(), bytes);
    return FSI_OK;
}

fsi_status load_array(Reader& r, void* dst, size_t bytes, bool dev, std::vector<char>& stage, cudaStream_t st) {
    if (bytes == 0) return FSI_OK;
    if (!dev) {
        r.get(dst, bytes);
        return r.ok ? FSI_OK : fail(FSI_EINVAL, "rom_load: file is truncated");
    }
    stage.resize(bytes);
    r.get(stage.data(), bytes);
    if (!r.ok) return fail(FSI_EINVAL, "rom_load: file is truncated");
    cudaError_t e = cudaMemcpyAsync(dst, stage.data(), bytes, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail(FSI_ECUDA, std::string("rom_load: ") + cudaGetErrorString(e));
    return FSI_OK;
}

fsi_status check_info(const fsi_rom_info& in) {
    if (!(in.nwin > 0 && in.kmax > 0 && in.nrhs > 0 && in.nrcv > 0 && in.n >= 0 && in.nshift_total >= 0))
        return fail(FSI_EINVAL, "rom: bad sizes in fsi_rom_info");
    return FSI_OK;
}

// The header (after the magic) of a ROM file; leaves the reader after the expansion points.
fsi_status read_head(Reader& r, fsi_rom_info& info, std::vector<double>& lo, std::vector<double>& hi,
                     std::vector<int32_t>& k, std::vector<int32_t>& ns, std::vector<double>& shifts) {
    char magic[8];
    if (std::fread(magic, 1, 8, r.f) != 8 || std::memcmp(magic, kMagic, 8) != 0)
        return fail(FSI_EINVAL, "rom_load: not a reduced-model file (bad magic)");
    int32_t h[6];
    int64_t n = 0;
    r.get(h, sizeof(h));
    r.get(&n, sizeof(n));
    if (!r.ok) return fail(FSI_EINVAL, "rom_load: file is truncated");
    if (h[0] != kVersion) return fail(FSI_EINVAL, "rom_load: unsupported file version " + std::to_string(h[0]));
    info.nwin = h[1];
    info.kmax = h[2];
    info.nrhs = h[3];
    info.nrcv = h[4];
    info.nshift_total = h[5];
    info.n = n;
    if (check_info(info) != FSI_OK || info.nwin > (1 << 20) || info.kmax > (1 << 20) || info.nshift_total > (1 << 24))
        return fail(FSI_EINVAL, "rom_load: corrupt header");
    lo.resize(info.nwin);
    hi.resize(info.nwin);
    k.resize(info.nwin);
    ns.resize(info.nwin);
    int64_t tot = 0;
    for (int w = 0; w < info.nwin; ++w) {
        r.get(&lo[w], sizeof(double));
        r.get(&hi[w], sizeof(double));
        r.get(&k[w], sizeof(int32_t));
        r.get(&ns[w], sizeof(int32_t));
        if (!r.ok) return fail(FSI_EINVAL, "rom_load: file is truncated");
        if (!(k[w] > 0 && k[w] <= info.kmax && ns[w] >= 0)) return fail(FSI_EINVAL, "rom_load: corrupt window table");
        tot += ns[w];
    }
    if (tot != info.nshift_total) return fail(FSI_EINVAL, "rom_load: corrupt window table");
    shifts.resize(size_t(tot));
    r.get(shifts.data(), sizeof(double) * size_t(tot));
    return r.ok ? FSI_OK : fail(FSI_EINVAL, "rom_load: file is truncated");
}

}  // namespace

}  // namespace fsi

using namespace fsi;

extern "C" {

fsi_status rom_save(const char* path, const fsi_rom_store* rom, void* stream) {
    if (!(path && rom)) return fail(FSI_EINVAL, "rom_save: NULL argument");
    const fsi_rom_info& in = rom->info;
    if (check_info(in) != FSI_OK) return FSI_EINVAL;
    if (!(rom->KR && rom->DR && rom->MR && rom->fR && rom->CR && rom->lo && rom->hi && rom->k && rom->nshift))
        return fail(FSI_EINVAL, "rom_save: NULL array");
    if (in.n > 0 && !rom->V) return fail(FSI_EINVAL, "rom_save: info.n > 0 needs the bases V");
    if (in.nshift_total > 0 && !rom->shifts_hz) return fail(FSI_EINVAL, "rom_save: NULL shifts_hz");
    int64_t tot = 0;
    for (int w = 0; w < in.nwin; ++w) {
        if (!(rom->k[w] > 0 && rom->k[w] <= in.kmax && rom->nshift[w] >= 0))
            return fail(FSI_EINVAL, "rom_save: window " + std::to_string(w) + " has k outside 1..kmax");
        tot += rom->nshift[w];
    }
    if (tot != in.nshift_total) return fail(FSI_EINVAL, "rom_save: nshift does not sum to nshift_total");
    FILE* f = std::fopen(path, "wb");
    if (!f) return fail(FSI_EINVAL, std::string("rom_save: cannot open ") + path);
    Writer w{f};
    bool ok = std::fwrite(kMagic, 1, 8, f) == 8;
    const int32_t h[6] = {kVersion, in.nwin, in.kmax, in.nrhs, in.nrcv, in.nshift_total};
    w.put(h, sizeof(h));
    w.put(&in.n, sizeof(in.n));
    for (int i = 0; i < in.nwin; ++i) {
        w.put(&rom->lo[i], sizeof(double));
        w.put(&rom->hi[i], sizeof(double));
        w.put(&rom->k[i], sizeof(int32_t));
        w.put(&rom->nshift[i], sizeof(int32_t));
    }
    if (tot > 0) w.put(rom->shifts_hz, sizeof(double) * size_t(tot));
    const bool dev = rom->on_device != 0;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    std::vector<char> stage;
    fsi_status s = FSI_OK;
    const size_t c16 = sizeof(fsi_c64);
    for (int i = 0; i < in.nwin && s == FSI_OK; ++i) {
        const size_t kk = size_t(rom->k[i]), km = size_t(in.kmax);
        s = save_array(w, rom->KR + i * km * km, kk * kk * c16, dev, stage, st);
        if (s == FSI_OK) s = save_array(w, rom->DR + i * km * km, kk * kk * c16, dev, stage, st);
        if (s == FSI_OK) s = save_array(w, rom->MR + i * km * km, kk * kk * c16, dev, stage, st);
        if (s == FSI_OK) s = save_array(w, rom->fR + i * km * in.nrhs, kk * in.nrhs * c16, dev, stage, st);
        if (s == FSI_OK) s = save_array(w, rom->CR + i * km * in.nrcv, kk * in.nrcv * c16, dev, stage, st);
        if (s == FSI_OK && in.n > 0) s = save_array(w, rom->V + i * km * in.n, kk * in.n * c16, dev, stage, st);
    }
    const uint64_t sum = w.sum.h;
    ok = ok && w.ok && std::fwrite(&sum, sizeof(sum), 1, f) == 1;
    ok = (std::fclose(f) == 0) && ok;
    if (s != FSI_OK) return s;
    if (!ok) return fail(FSI_EINVAL, std::string("rom_save: write failed for ") + path);
    return FSI_OK;
}

fsi_status rom_file_info(const char* path, fsi_rom_info* info) {
    if (!(path && info)) return fail(FSI_EINVAL, "rom_file_info: NULL argument");
    FILE* f = std::fopen(path, "rb");
    if (!f) return fail(FSI_EINVAL, std::string("rom_file_info: cannot open ") + path);
    Reader r{f};
    std::vector<double> lo, hi, shifts;
    std::vector<int32_t> k, ns;
    fsi_status s = read_head(r, *info, lo, hi, k, ns, shifts);
    std::fclose(f);
    return s;
}

fsi_status rom_load(const char* path, fsi_rom_store* rom, void* stream) {
    if (!(path && rom)) return fail(FSI_EINVAL, "rom_load: NULL argument");
    FILE* f = std::fopen(path, "rb");
    if (!f) return fail(FSI_EINVAL, std::string("rom_load: cannot open ") + path);
    Reader r{f};
    fsi_rom_info info{};
    std::vector<double> lo, hi, shifts;
    std::vector<int32_t> k, ns;
    fsi_status s = read_head(r, info, lo, hi, k, ns, shifts);
    const fsi_rom_info want = rom->info;   // a copy: rom->info is overwritten on success
    if (s == FSI_OK && !(want.nwin >= info.nwin && want.kmax >= info.kmax && want.nrhs == info.nrhs &&
                         want.nrcv == info.nrcv && want.nshift_total >= info.nshift_total &&
                         (info.n == 0 || want.n == info.n)))
        s = fail(FSI_EINVAL, "rom_load: buffers described by rom->info are smaller than the file's model "
                             "(read the sizes with rom_file_info)");
    if (s == FSI_OK && !(rom->KR && rom->DR && rom->MR && rom->fR && rom->CR && rom->lo && rom->hi && rom->k &&
                         rom->nshift && (info.nshift_total == 0 || rom->shifts_hz) && (info.n == 0 || rom->V)))
        s = fail(FSI_EINVAL, "rom_load: NULL array");
    const bool dev = rom->on_device != 0;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    std::vector<char> stage;
    const size_t c16 = sizeof(fsi_c64);
    // windows go to the slots of the caller's kmax
    const size_t km = size_t(want.kmax);
    for (int i = 0; i < info.nwin && s == FSI_OK; ++i) {
        const size_t kk = size_t(k[i]);
        s = load_array(r, rom->KR + i * km * km, kk * kk * c16, dev, stage, st);
        if (s == FSI_OK) s = load_array(r, rom->DR + i * km * km, kk * kk * c16, dev, stage, st);
        if (s == FSI_OK) s = load_array(r, rom->MR + i * km * km, kk * kk * c16, dev, stage, st);
        if (s == FSI_OK) s = load_array(r, rom->fR + i * km * info.nrhs, kk * info.nrhs * c16, dev, stage, st);
        if (s == FSI_OK) s = load_array(r, rom->CR + i * km * info.nrcv, kk * info.nrcv * c16, dev, stage, st);
        if (s == FSI_OK && info.n > 0)
            s = load_array(r, rom->V + i * km * size_t(info.n), kk * size_t(info.n) * c16, dev, stage, st);
    }
    if (s == FSI_OK) {
        const uint64_t expect = r.sum.h;
        uint64_t got = 0;
        if (std::fread(&got, sizeof(got), 1, f) != 1) s = fail(FSI_EINVAL, "rom_load: file is truncated");
        else if (got != expect) s = fail(FSI_EINVAL, "rom_load: checksum mismatch (file corrupt)");
    }
    std::fclose(f);
    if (s != FSI_OK) return s;
    rom->info = info;
    rom->info.kmax = want.kmax;   // the slot layout of the caller's buffers
    for (int i = 0; i < info.nwin; ++i) {
        rom->lo[i] = lo[i];
        rom->hi[i] = hi[i];
        rom->k[i] = k[i];
        rom->nshift[i] = ns[i];
    }
    if (!shifts.empty()) std::memcpy(rom->shifts_hz, shifts.data(), sizeof(double) * shifts.size());
    return FSI_OK;
}

fsi_status rom_check_resolve_workspace(const fsi_dims* dims, int k, int nrhs, int nrcv, int batch,
                                       const fsi_solve_opts* full, size_t* bytes) {
    if (!(dims && full && bytes && k > 0 && nrhs > 0 && nrcv > 0 && batch > 0))
        return fail(FSI_EINVAL, "rom_check_resolve_workspace: bad arguments");
    size_t a = 0, b = 0;
    fsi_status s = rom_residual_check_workspace(dims, k, nrhs, batch, &a);
    if (s != FSI_OK) return s;
    fsi_solve_opts o = *full;
    o.batch = std::max(1, std::min(o.batch, batch));
    o.host_io = 0;
    s = frf_sweep_workspace(dims, &o, nrhs, nrcv, &b);
    if (s != FSI_OK) return s;
    const size_t out = align_up(size_t(batch) * nrcv * nrhs * (sizeof(fsi_c64) + sizeof(double)));
    *bytes = std::max(a, align_up(b) + out);
    return FSI_OK;
}

fsi_status rom_check_resolve(const fsi_dims* dims, const void* d_model, const fsi_c64* V, int k, const fsi_c64* KR,
                             const fsi_c64* DR, const fsi_c64* MR, const fsi_c64* fR, const fsi_c64* F, int nrhs,
                             const int32_t* rcv, int nrcv, const double* f_hz, int nf, int batch, double res_tol,
                             const fsi_solve_opts* full, void* ws, size_t ws_bytes, fsi_c64* p_out, double* spl_out,
                             double* relres_out, int32_t* resolved_out, int* n_resolved, void* stream) {
    if (!(dims && d_model && V && KR && DR && MR && fR && F && rcv && f_hz && full && ws && p_out && n_resolved))
        return fail(FSI_EINVAL, "rom_check_resolve: NULL argument");
    if (!(k > 0 && nrhs > 0 && nrhs <= 8 && nrcv > 0 && nf > 0 && batch > 0 && res_tol >= 0.0))
        return fail(FSI_EINVAL, "rom_check_resolve: bad sizes or tolerance");
    if (full->host_io) return fail(FSI_EINVAL, "rom_check_resolve: full->host_io must be 0 (device buffers)");
    const int bt = std::min(batch, nf);
    size_t need = 0;
    fsi_status s = rom_check_resolve_workspace(dims, k, nrhs, nrcv, bt, full, &need);
    if (s != FSI_OK) return s;
    if (ws_bytes < need) return fail(FSI_ENOMEM, "rom_check_resolve: workspace too small");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // 1. the judge: full-order FP64 residual of every lifted reduced solution
    std::vector<double> rel(size_t(nf) * nrhs);
    s = rom_residual_check(dims, d_model, V, k, KR, DR, MR, fR, F, nrhs, f_hz, nf, bt, ws, ws_bytes, rel.data(),
                           stream);
    if (s != FSI_OK) return s;
    std::vector<int> bad;
    for (int i = 0; i < nf; ++i) {
        double r = 0.0;
        for (int c = 0; c < nrhs; ++c) {
            const double v = rel[size_t(i) * nrhs + c];
            r = std::isfinite(v) ? std::max(r, v) : INFINITY;
        }
        if (r > res_tol) bad.push_back(i);
        if (resolved_out) resolved_out[i] = r > res_tol ? 1 : 0;
    }
    if (relres_out) std::memcpy(relres_out, rel.data(), sizeof(double) * rel.size());
    *n_resolved = int(bad.size());
    // 2. the fallback: failing frequencies at full order, their outputs over the reduced ones
    fsi_solve_opts o = *full;
    o.batch = std::max(1, std::min(o.batch, bt));
    o.host_io = 0;
    size_t sweep_bytes = 0;
    s = frf_sweep_workspace(dims, &o, nrhs, nrcv, &sweep_bytes);
    if (s != FSI_OK) return s;
    sweep_bytes = align_up(sweep_bytes);
    fsi_c64* pt = reinterpret_cast<fsi_c64*>(static_cast<char*>(ws) + sweep_bytes);
    double* splt = reinterpret_cast<double*>(pt + size_t(bt) * nrcv * nrhs);
    const size_t row = size_t(nrcv) * nrhs;
    std::vector<double> fb;
    bool noconv = false;
    for (size_t b0 = 0; b0 < bad.size(); b0 += size_t(bt)) {
        const int nb = int(std::min(bad.size() - b0, size_t(bt)));
        fb.assign(nb, 0.0);
        for (int j = 0; j < nb; ++j) fb[j] = f_hz[bad[b0 + j]];
        fsi_sweep_stats stats{};
        s = frf_sweep_full(dims, d_model, fb.data(), nb, F, nrhs, rcv, nrcv, &o, ws, sweep_bytes, pt, splt, nullptr,
                           nullptr, &stats, stream);
        if (s == FSI_ENOCONV) noconv = true;   // results are written; reported at the end
        else if (s != FSI_OK) return s;
        for (int j = 0; j < nb; ++j) {
            const int i = bad[b0 + j];
            cudaError_t e = cudaMemcpyAsync(p_out + size_t(i) * row, pt + size_t(j) * row, sizeof(fsi_c64) * row,
                                            cudaMemcpyDeviceToDevice, st);
            if (e == cudaSuccess && spl_out)
                e = cudaMemcpyAsync(spl_out + size_t(i) * row, splt + size_t(j) * row, sizeof(double) * row,
                                    cudaMemcpyDeviceToDevice, st);
            if (e != cudaSuccess) return fail(FSI_ECUDA, std::string("rom_check_resolve: ") + cudaGetErrorString(e));
        }
    }
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail(FSI_ECUDA, std::string("rom_check_resolve: ") + cudaGetErrorString(e));
    if (noconv) return fail(FSI_ENOCONV, "rom_check_resolve: a full-order re-solve did not reach its tolerance");
    return FSI_OK;
}

}  // extern "C"
