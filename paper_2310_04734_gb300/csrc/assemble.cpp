// Host assembly of the coupled shell-cavity model (paper Sec. 2, Eq. 1-3;
// coupling matrix Eq. 5; complex stiffness and the damping matrix of Eq. 8).
//
// The uniform structured mesh lets every element matrix be written in closed
// form:
//   * trilinear pressure hexahedron: tensor products of the 1-D linear element
//     stiffness k1(h) = [1 -1; -1 1]/h and mass m1(h) = h/6 [2 1; 1 2]:
//       Kf = kx(x)my(x)mz + mx(x)ky(x)mz + mx(x)my(x)kz,  Mf = mx(x)my(x)mz / c^2
//   * wall face (coupling, floor impedance): m1(L)(x)m1(hz)
//   * rectangular Reissner-Mindlin plate (w, beta_s, beta_z), bending with
//     2x2 Gauss points, transverse shear by the MITC4 edge-midpoint tying
//     written directly on the rectangle's edges, consistent mass in tensor form.
// Coupling: K_sf = -C, M_fs = rho C^T, w the wall displacement pointing out of
// the cavity (the paper's Eq. 5 carries rho_f and Eq. 2 carries rho again in
// front of C^T; the density is applied once, in M).  Floor: D = (rho/Z) m_face.
// Shell ends (slabs 0 and nz-1) are simply supported: w rows and columns are
// cleared except the stiffness diagonal.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <sstream>

#include "fsi_internal.h"

namespace fsi {

namespace {

using cplx = std::complex<double>;

struct Entry {
    int32_t col;
    cplx k;
    double m;
    cplx d;
};

class Builder {
   public:
    explicit Builder(int64_t n) : rows_(n) {}
    void add(int64_t r, int64_t c, cplx k, double m, cplx d) {
        auto& row = rows_[r];
        for (auto& e : row) {
            if (e.col == c) {
                e.k += k;
                e.m += m;
                e.d += d;
                return;
            }
        }
        row.push_back(Entry{static_cast<int32_t>(c), k, m, d});
    }
    std::vector<std::vector<Entry>>& rows() { return rows_; }

   private:
    std::vector<std::vector<Entry>> rows_;
};

void k1(double h, double out[2][2]) {
    out[0][0] = out[1][1] = 1.0 / h;
    out[0][1] = out[1][0] = -1.0 / h;
}
void m1(double h, double out[2][2]) {
    out[0][0] = out[1][1] = h / 3.0;
    out[0][1] = out[1][0] = h / 6.0;
}

// Rectangular MITC4 plate, nodes (0,0), (a,0), (a,c), (0,c); DoF 3*node + {w, bs, bz}.
void plate_rect(double a, double c, double E, double nu, double rho, double t, double Ke[12][12],
                double Me[12][12]) {
    const double Dfac = E * t * t * t / (12.0 * (1.0 - nu * nu));
    const double Db[3][3] = {{Dfac, Dfac * nu, 0.0}, {Dfac * nu, Dfac, 0.0}, {0.0, 0.0, Dfac * (1.0 - nu) / 2.0}};
    const double Gs = 5.0 / 6.0 * E / (2.0 * (1.0 + nu)) * t;
    const double gp = 1.0 / std::sqrt(3.0);
    const int nxi[4] = {-1, 1, 1, -1}, neta[4] = {-1, -1, 1, 1};
    std::memset(Ke, 0, sizeof(double) * 144);
    std::memset(Me, 0, sizeof(double) * 144);
    // edge shear rows: gamma_s on edges z=0 (nodes 0,1) and z=c (nodes 3,2);
    // gamma_z on edges s=0 (nodes 0,3) and s=a (nodes 1,2)
    double gsA[12] = {0}, gsC[12] = {0}, gzD[12] = {0}, gzB[12] = {0};
    gsA[0] = -1.0 / a; gsA[3] = 1.0 / a; gsA[1] = 0.5; gsA[4] = 0.5;
    gsC[9] = -1.0 / a; gsC[6] = 1.0 / a; gsC[10] = 0.5; gsC[7] = 0.5;
    gzD[0] = -1.0 / c; gzD[9] = 1.0 / c; gzD[2] = 0.5; gzD[11] = 0.5;
    gzB[3] = -1.0 / c; gzB[6] = 1.0 / c; gzB[5] = 0.5; gzB[8] = 0.5;
    const double detJ = a * c / 4.0;
    for (int gi = 0; gi < 2; ++gi) {
        for (int gj = 0; gj < 2; ++gj) {
            const double xi = gi ? gp : -gp, eta = gj ? gp : -gp;
            double Bb[3][12] = {{0}};
            for (int n = 0; n < 4; ++n) {
                const double dNs = nxi[n] * (1.0 + neta[n] * eta) / 4.0 * (2.0 / a);
                const double dNz = neta[n] * (1.0 + nxi[n] * xi) / 4.0 * (2.0 / c);
                Bb[0][3 * n + 1] = dNs;
                Bb[1][3 * n + 2] = dNz;
                Bb[2][3 * n + 1] = dNz;
                Bb[2][3 * n + 2] = dNs;
            }
            double Bs[2][12];
            for (int q = 0; q < 12; ++q) {
                Bs[0][q] = 0.5 * (1.0 - eta) * gsA[q] + 0.5 * (1.0 + eta) * gsC[q];
                Bs[1][q] = 0.5 * (1.0 - xi) * gzD[q] + 0.5 * (1.0 + xi) * gzB[q];
            }
            for (int p = 0; p < 12; ++p) {
                for (int q = 0; q < 12; ++q) {
                    double s = 0.0;
                    for (int i = 0; i < 3; ++i)
                        for (int j = 0; j < 3; ++j) s += Bb[i][p] * Db[i][j] * Bb[j][q];
                    s += Gs * (Bs[0][p] * Bs[0][q] + Bs[1][p] * Bs[1][q]);
                    Ke[p][q] += s * detJ;
                }
            }
        }
    }
    // consistent mass: (m1(a) (x) m1(c)) per DoF component
    double ma[2][2], mc[2][2];
    m1(a, ma);
    m1(c, mc);
    const int bs[4] = {0, 1, 1, 0}, bz[4] = {0, 0, 1, 1};
    const double md[3] = {rho * t, rho * t * t * t / 12.0, rho * t * t * t / 12.0};
    for (int p = 0; p < 4; ++p)
        for (int q = 0; q < 4; ++q)
            for (int d = 0; d < 3; ++d) Me[3 * p + d][3 * q + d] = md[d] * ma[bs[p]][bs[q]] * mc[bz[p]][bz[q]];
}

}  // namespace

fsi_status validate_desc(const fsi_model_desc& d) {
    std::ostringstream msg;
    if (d.nx < 3 || d.ny < 3 || d.nz < 3) msg << "nx, ny, nz must be >= 3; ";
    if (!(d.Lx > 0 && d.Ly > 0 && d.Lz > 0)) msg << "box lengths must be positive; ";
    if (!(d.c > 0 && d.rho > 0 && d.E > 0 && d.rho_s > 0 && d.t > 0)) msg << "material constants must be positive; ";
    if (!(d.nu > -1.0 && d.nu < 0.5)) msg << "nu out of range; ";
    if (!d.eta || !(d.n_eta == 1 || d.n_eta == d.nz - 1)) msg << "eta must have 1 or nz-1 entries; ";
    if (d.has_floor && d.Z_re == 0.0 && d.Z_im == 0.0) msg << "floor impedance must be nonzero; ";
    const int64_t nr = 2LL * (d.nx - 1) + 2LL * (d.ny - 1);
    const int64_t b = int64_t(d.nx) * d.ny + 3 * nr;
    if (b * int64_t(d.nz) >= (int64_t(1) << 31)) msg << "model too large for 32-bit indices; ";
    if (!msg.str().empty()) {
        set_error("fsi_model_desc: " + msg.str());
        return FSI_EINVAL;
    }
    return FSI_OK;
}

ModelLayout model_layout(const fsi_dims& d) {
    ModelLayout L{};
    size_t off = 0;
    auto put = [&](size_t bytes) {
        size_t o = align_up(off);
        off = o + bytes;
        return o;
    };
    L.rowptr = put(sizeof(int32_t) * (d.n + 1));
    L.col = put(sizeof(int32_t) * d.nnz);
    L.K = put(sizeof(fsi_c64) * d.nnz);
    L.M = put(sizeof(double) * d.nnz);
    L.D = put(sizeof(fsi_c64) * d.nnz);
    L.kdiag = put(sizeof(double) * d.n);
    L.cbase = put(sizeof(double) * d.n);
    L.rbase = put(sizeof(double) * d.n);
    L.total = align_up(off);
    return L;
}

fsi_status assemble_host(const fsi_model_desc& d, HostModel& out) {
    fsi_status st = validate_desc(d);
    if (st != FSI_OK) return st;
    const int nx = d.nx, ny = d.ny, nz = d.nz;
    const int npl = nx * ny;
    const int nr = 2 * (nx - 1) + 2 * (ny - 1);
    const int b = npl + 3 * nr;
    const int64_t n = int64_t(b) * nz;
    const double hx = d.Lx / (nx - 1), hy = d.Ly / (ny - 1), hz = d.Lz / (nz - 1);

    // ring node grid positions, counter-clockwise from (0, 0)
    std::vector<int> ri(nr), rj(nr);
    {
        int i = 0, j = 0, r = 0;
        const int di[4] = {1, 0, -1, 0}, dj[4] = {0, 1, 0, -1};
        const int len[4] = {nx - 1, ny - 1, nx - 1, ny - 1};
        for (int side = 0; side < 4; ++side)
            for (int s = 0; s < len[side]; ++s) {
                ri[r] = i;
                rj[r] = j;
                ++r;
                i += di[side];
                j += dj[side];
            }
    }
    auto pdof = [&](int i, int j, int k) { return int64_t(k) * b + i + int64_t(nx) * j; };
    auto sdof = [&](int r, int k, int comp) { return int64_t(k) * b + npl + 3 * r + comp; };

    Builder B(n);
    const cplx zero(0.0, 0.0);

    // ---- cavity: trilinear hexahedra
    {
        double kx[2][2], ky[2][2], kz[2][2], mx[2][2], my[2][2], mz[2][2];
        k1(hx, kx); k1(hy, ky); k1(hz, kz);
        m1(hx, mx); m1(hy, my); m1(hz, mz);
        const double ic2 = 1.0 / (d.c * d.c);
        for (int k = 0; k < nz - 1; ++k)
            for (int j = 0; j < ny - 1; ++j)
                for (int i = 0; i < nx - 1; ++i)
                    for (int a = 0; a < 8; ++a) {
                        const int ax = a & 1, ay = (a >> 1) & 1, az = (a >> 2) & 1;
                        const int64_t ra = pdof(i + ax, j + ay, k + az);
                        for (int c = 0; c < 8; ++c) {
                            const int cx = c & 1, cy = (c >> 1) & 1, cz = (c >> 2) & 1;
                            const double kv = kx[ax][cx] * my[ay][cy] * mz[az][cz] +
                                              mx[ax][cx] * ky[ay][cy] * mz[az][cz] +
                                              mx[ax][cx] * my[ay][cy] * kz[az][cz];
                            const double mv = mx[ax][cx] * my[ay][cy] * mz[az][cz] * ic2;
                            B.add(ra, pdof(i + cx, j + cy, k + cz), cplx(kv, 0.0), mv, zero);
                        }
                    }
    }

    // ---- shell ring (developed flat plate, periodic in s) and wall coupling
    {
        double Ke[12][12], Me[12][12];
        double mzz[2][2];
        m1(hz, mzz);
        for (int r = 0; r < nr; ++r) {
            const int r2 = (r + 1) % nr;
            const double L = (ri[r] != ri[r2]) ? hx : hy;
            plate_rect(L, hz, d.E, d.nu, d.rho_s, d.t, Ke, Me);
            double ms[2][2];
            m1(L, ms);
            for (int k = 0; k < nz - 1; ++k) {
                const double eta = d.n_eta == 1 ? d.eta[0] : d.eta[k];
                const cplx damp(1.0, eta);
                const int nodes_r[4] = {r, r2, r2, r};
                const int nodes_k[4] = {k, k, k + 1, k + 1};
                for (int p = 0; p < 4; ++p)
                    for (int dp = 0; dp < 3; ++dp) {
                        const int64_t row = sdof(nodes_r[p], nodes_k[p], dp);
                        for (int q = 0; q < 4; ++q)
                            for (int dq = 0; dq < 3; ++dq) {
                                const double kv = Ke[3 * p + dp][3 * q + dq];
                                const double mv = Me[3 * p + dp][3 * q + dq];
                                if (kv == 0.0 && mv == 0.0) continue;
                                B.add(row, sdof(nodes_r[q], nodes_k[q], dq), damp * kv, mv, zero);
                            }
                    }
                // coupling through the shared wall face: C_ab = m1(L)[as][bs] * m1(hz)[az][bz]
                for (int as = 0; as < 2; ++as)
                    for (int az = 0; az < 2; ++az) {
                        const int ra = as ? r2 : r;
                        const int64_t w = sdof(ra, k + az, 0);
                        const int64_t pw = pdof(ri[ra], rj[ra], k + az);
                        for (int bs2 = 0; bs2 < 2; ++bs2)
                            for (int bz = 0; bz < 2; ++bz) {
                                const int rb = bs2 ? r2 : r;
                                const double cv = ms[as][bs2] * mzz[az][bz];
                                const int64_t p = pdof(ri[rb], rj[rb], k + bz);
                                const int64_t wb = sdof(rb, k + bz, 0);
                                B.add(w, p, cplx(-cv, 0.0), 0.0, zero);     // K_sf = -C
                                B.add(pw, wb, zero, d.rho * cv, zero);      // M_fs = rho C^T
                            }
                    }
            }
        }
    }

    // ---- floor impedance on y = 0: D = (rho / Z) m1(hx) (x) m1(hz)
    if (d.has_floor) {
        const cplx beta = d.rho / cplx(d.Z_re, d.Z_im);
        double mx[2][2], mz[2][2];
        m1(hx, mx);
        m1(hz, mz);
        for (int k = 0; k < nz - 1; ++k)
            for (int i = 0; i < nx - 1; ++i)
                for (int ax = 0; ax < 2; ++ax)
                    for (int az = 0; az < 2; ++az)
                        for (int cx = 0; cx < 2; ++cx)
                            for (int cz = 0; cz < 2; ++cz)
                                B.add(pdof(i + ax, 0, k + az), pdof(i + cx, 0, k + cz), zero, 0.0,
                                      beta * (mx[ax][cx] * mz[az][cz]));
    }

    // ---- simply supported shell ends: clear w rows/cols on slabs 0 and nz-1,
    // keep the stiffness diagonal
    std::vector<char> fixed(n, 0);
    for (int r = 0; r < nr; ++r) {
        fixed[sdof(r, 0, 0)] = 1;
        fixed[sdof(r, nz - 1, 0)] = 1;
    }

    auto& rows = B.rows();
    out.dims.n = n;
    out.dims.b = b;
    out.dims.nz = nz;
    out.dims.n_press_slab = npl;
    out.dims.n_ring = nr;
    out.dims.rho = d.rho;
    out.rowptr.assign(n + 1, 0);
    out.col.clear();
    out.K.clear();
    out.M.clear();
    out.D.clear();
    out.kdiag.assign(n, 0.0);
    for (int64_t r = 0; r < n; ++r) {
        auto& row = rows[r];
        std::sort(row.begin(), row.end(), [](const Entry& x, const Entry& y) { return x.col < y.col; });
        for (const auto& e : row) {
            if (fixed[r] || fixed[e.col]) {
                if (!(fixed[r] && e.col == r)) continue;
                out.col.push_back(e.col);
                out.K.push_back(fsi_c64{e.k.real(), e.k.imag()});
                out.M.push_back(0.0);
                out.D.push_back(fsi_c64{0.0, 0.0});
            } else {
                out.col.push_back(e.col);
                out.K.push_back(fsi_c64{e.k.real(), e.k.imag()});
                out.M.push_back(e.m);
                out.D.push_back(fsi_c64{e.d.real(), e.d.imag()});
            }
            if (e.col == r) out.kdiag[r] = std::abs(e.k);
        }
        out.rowptr[r + 1] = static_cast<int32_t>(out.col.size());
        std::vector<Entry>().swap(row);
    }
    out.dims.nnz = static_cast<int64_t>(out.col.size());
    out.dims.model_bytes = model_layout(out.dims).total;
    for (int64_t r = 0; r < n; ++r) {
        if (!(out.kdiag[r] > 0.0)) {
            set_error("assembly produced a zero stiffness diagonal");
            return FSI_EINVAL;
        }
    }
    return FSI_OK;
}

}  // namespace fsi
