"""Oracle FE assembly (TEST INFRASTRUCTURE ONLY; see package docstring).

Everything here is written as the textbook isoparametric recipe: shape
functions on the reference element, Jacobian, Gauss quadrature, scatter into
global sparse matrices.  Nothing is specialised to the uniform mesh.

Physics (paper Sec. 2, Eq. 1-3, and Sec. 3.3, Eq. 8 with the complex stiffness
K(w) = K^(1 + i eta) stated after it):

* cavity, Helmholtz in pressure p:  Kf = int grad N . grad N dV,
  Mf = (1/c^2) int N N dV                                       (Eq. 1)
* shell ring, Reissner-Mindlin plate with DoFs (w, beta_s, beta_z) per node,
  bending + transverse shear (MITC4 assumed shear, Bathe-Dvorkin 1985),
  stiffness multiplied by (1 + i eta_layer)                     (Sec. 2, Sec. 3.3)
* coupling, conforming: C_ab = int_Gamma N^s_a N^f_b dGamma with w the
  wall-normal displacement pointing out of the cavity; K gets -C in the
  shell rows and M gets rho*C^T in the fluid rows               (Eq. 2, Eq. 5)
  (the paper puts rho_f inside Eq. 5 *and* in front of C^T in Eq. 2; the
  density is counted once, in M.)
* locally reacting floor impedance Z on y = 0: D = (rho/Z) int N N dGamma,
  entering as +i w D                                            (Eq. 8)

The global system is A(w) = K + i w D - w^2 M with slab-major DoF ordering.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import List, Tuple

import numpy as np
import scipy.sparse as sp

G2 = (-1.0 / np.sqrt(3.0), 1.0 / np.sqrt(3.0))   # 2-point Gauss abscissae, unit weights

# reference-node signs of the 8-node hexahedron and the 4-node quadrilateral
HEX_NODES = np.array([[-1, -1, -1], [1, -1, -1], [1, 1, -1], [-1, 1, -1],
                      [-1, -1, 1], [1, -1, 1], [1, 1, 1], [-1, 1, 1]], dtype=float)
QUAD_NODES = np.array([[-1, -1], [1, -1], [1, 1], [-1, 1]], dtype=float)


# --------------------------------------------------------------------------- elements
def hex8_shape(xi, eta, zeta):
    """Trilinear shape functions and their reference derivatives at one point."""
    N = np.empty(8)
    dN = np.empty((8, 3))
    for a, (sa, ta, ua) in enumerate(HEX_NODES):
        fx, fy, fz = 1 + sa * xi, 1 + ta * eta, 1 + ua * zeta
        N[a] = fx * fy * fz / 8.0
        dN[a, 0] = sa * fy * fz / 8.0
        dN[a, 1] = ta * fx * fz / 8.0
        dN[a, 2] = ua * fx * fy / 8.0
    return N, dN


def hex8_matrices(X: np.ndarray):
    """Element Laplacian and mass for an 8-node hexahedron with node coordinates X (8x3).

    Returns (Ke, Me) with Ke = int grad N grad N^T dV and Me = int N N^T dV, by
    2x2x2 Gauss quadrature (exact for the trilinear element on a parallelepiped).
    """
    Ke = np.zeros((8, 8))
    Me = np.zeros((8, 8))
    for xi in G2:
        for eta in G2:
            for zeta in G2:
                N, dN = hex8_shape(xi, eta, zeta)
                J = dN.T @ X                     # J[r, c] = d x_c / d xi_r
                detJ = np.linalg.det(J)
                gradN = np.linalg.solve(J, dN.T).T   # rows: dN_a/dx
                Ke += gradN @ gradN.T * detJ
                Me += np.outer(N, N) * detJ
    return Ke, Me


def quad4_shape(xi, eta):
    N = np.empty(4)
    dN = np.empty((4, 2))
    for a, (sa, ta) in enumerate(QUAD_NODES):
        N[a] = (1 + sa * xi) * (1 + ta * eta) / 4.0
        dN[a, 0] = sa * (1 + ta * eta) / 4.0
        dN[a, 1] = ta * (1 + sa * xi) / 4.0
    return N, dN


def quad4_surface_mass(X: np.ndarray):
    """int_Gamma N N^T dGamma over a 4-node surface quad embedded in 3-D (X: 4x3)."""
    Me = np.zeros((4, 4))
    for xi in G2:
        for eta in G2:
            N, dN = quad4_shape(xi, eta)
            t1 = dN[:, 0] @ X
            t2 = dN[:, 1] @ X
            dA = np.linalg.norm(np.cross(t1, t2))
            Me += np.outer(N, N) * dA
    return Me


def mitc4_plate(X2: np.ndarray, E: float, nu: float, rho: float, t: float):
    """Reissner-Mindlin plate element (4 nodes, DoFs w, beta_s, beta_z per node).

    X2: node coordinates (4x2) in the plate plane (s, z).  Kinematics: in-plane
    displacement zeta*beta, curvatures (d beta_s/ds, d beta_z/dz, d beta_s/dz +
    d beta_z/ds), transverse shear gamma = grad w + beta.  Transverse shear uses
    the MITC4 assumed covariant strains: gamma_xi tied at the edge midpoints
    (0, -1) and (0, +1) and interpolated linearly in eta; gamma_eta tied at
    (-1, 0) and (+1, 0) and interpolated linearly in xi.  Returns (Ke, Me) of
    size 12x12 with DoF order [w1, bs1, bz1, w2, ...].
    """
    Db = E * t ** 3 / (12.0 * (1.0 - nu ** 2)) * np.array(
        [[1.0, nu, 0.0], [nu, 1.0, 0.0], [0.0, 0.0, (1.0 - nu) / 2.0]])
    G = E / (2.0 * (1.0 + nu))
    ks = 5.0 / 6.0
    Ds = ks * G * t

    def covariant_shear_rows(xi, eta):
        """Rows mapping element DoFs to (gamma_xi, gamma_eta) covariant shear at a point."""
        N, dN = quad4_shape(xi, eta)
        J = dN.T @ X2                 # J[r, c] = d x_c / d xi_r
        B = np.zeros((2, 12))
        for a in range(4):
            for r in range(2):
                B[r, 3 * a + 0] = dN[a, r]                 # dw/dxi_r
                B[r, 3 * a + 1] = N[a] * J[r, 0]           # beta_s * ds/dxi_r
                B[r, 3 * a + 2] = N[a] * J[r, 1]           # beta_z * dz/dxi_r
        return B

    tie_A = covariant_shear_rows(0.0, -1.0)[0]
    tie_C = covariant_shear_rows(0.0, 1.0)[0]
    tie_D = covariant_shear_rows(-1.0, 0.0)[1]
    tie_B = covariant_shear_rows(1.0, 0.0)[1]

    Ke = np.zeros((12, 12))
    Me = np.zeros((12, 12))
    mass_diag = np.array([rho * t, rho * t ** 3 / 12.0, rho * t ** 3 / 12.0])
    for xi in G2:
        for eta in G2:
            N, dN = quad4_shape(xi, eta)
            J = dN.T @ X2
            detJ = np.linalg.det(J)
            dNx = np.linalg.solve(J, dN.T).T      # dN_a/ds, dN_a/dz
            Bb = np.zeros((3, 12))
            for a in range(4):
                Bb[0, 3 * a + 1] = dNx[a, 0]
                Bb[1, 3 * a + 2] = dNx[a, 1]
                Bb[2, 3 * a + 1] = dNx[a, 1]
                Bb[2, 3 * a + 2] = dNx[a, 0]
            Ke += Bb.T @ Db @ Bb * detJ
            gxi = 0.5 * (1 - eta) * tie_A + 0.5 * (1 + eta) * tie_C
            geta = 0.5 * (1 - xi) * tie_D + 0.5 * (1 + xi) * tie_B
            Bcov = np.vstack([gxi, geta])
            Bs = np.linalg.solve(J, Bcov)          # Cartesian shear = J^-1 covariant
            Ke += Bs.T @ Bs * Ds * detJ
            Nm = np.zeros((3, 12))
            for a in range(4):
                for d in range(3):
                    Nm[d, 3 * a + d] = N[a]
            Me += Nm.T @ np.diag(mass_diag) @ Nm * detJ
    return Ke, Me


# --------------------------------------------------------------------------- mesh
def ring_nodes(nx: int, ny: int) -> List[Tuple[int, int]]:
    """(i, j) grid position of each shell ring node, counter-clockwise from (0, 0)."""
    out = []
    i, j = 0, 0
    for di, dj, steps in ((1, 0, nx - 1), (0, 1, ny - 1), (-1, 0, nx - 1), (0, -1, ny - 1)):
        for _ in range(steps):
            out.append((i, j))
            i += di
            j += dj
    return out


@dataclass
class Assembled:
    spec: object
    K: sp.csr_matrix     # complex128
    M: sp.csr_matrix     # float64
    D: sp.csr_matrix     # complex128
    b: int
    nz: int
    n: int
    is_fluid: np.ndarray   # bool mask of pressure DoFs

    def A(self, omega: float) -> sp.csr_matrix:
        """A(w) = K + i w D - w^2 M (Eq. 8)."""
        return (self.K + 1j * omega * self.D - omega ** 2 * self.M).tocsr()


class Numbering:
    """Slab-major DoF numbering: slab k holds nx*ny pressure DoFs (i + nx*j), then
    (w, beta_s, beta_z) for each ring node."""

    def __init__(self, spec):
        self.nx, self.ny, self.nz = spec.nx, spec.ny, spec.nz
        self.ring = ring_nodes(spec.nx, spec.ny)
        self.nr = len(self.ring)
        self.npl = spec.nx * spec.ny
        self.b = self.npl + 3 * self.nr
        self.n = self.b * self.nz

    def p(self, i, j, k):
        return k * self.b + i + self.nx * j

    def s(self, r, k, comp):
        return k * self.b + self.npl + 3 * r + comp


def assemble(spec) -> Assembled:
    """Assemble K (complex), M (real), D (complex) of the coupled model."""
    num = Numbering(spec)
    hx = spec.Lx / (spec.nx - 1)
    hy = spec.Ly / (spec.ny - 1)
    hz = spec.Lz / (spec.nz - 1)
    Kr, Kc, Kv = [], [], []
    Mr, Mc, Mv = [], [], []
    Dr, Dc, Dv = [], [], []

    def put(R, Cc, V, rows, cols, mat):
        rows = np.asarray(rows)
        cols = np.asarray(cols)
        R.append(np.repeat(rows, len(cols)))
        Cc.append(np.tile(cols, len(rows)))
        V.append(np.asarray(mat).ravel())

    # Element matrices depend only on the element's shape; on a uniform mesh most
    # elements are translates of each other, so results are memoised by the node
    # coordinates relative to the first node (the recipe itself is unchanged).
    memo = {}

    def cached(kind, X, fn):
        key = (kind, tuple(np.round((X - X[0]).ravel(), 12)))
        if key not in memo:
            memo[key] = fn(X)
        return memo[key]

    def xyz(i, j, k):
        return np.array([i * hx, j * hy, k * hz])

    # ---- cavity (Eq. 1, Omega_4 analogue)
    for k in range(spec.nz - 1):
        for j in range(spec.ny - 1):
            for i in range(spec.nx - 1):
                nodes = []
                for (sa, ta, ua) in HEX_NODES:
                    nodes.append((i + (sa > 0), j + (ta > 0), k + (ua > 0)))
                X = np.array([xyz(*nd) for nd in nodes])
                Ke, Me = cached('hex', X, hex8_matrices)
                dofs = [num.p(*nd) for nd in nodes]
                put(Kr, Kc, Kv, dofs, dofs, Ke.astype(complex))
                put(Mr, Mc, Mv, dofs, dofs, Me / spec.c ** 2)

    # ---- shell ring (developed flat plate, periodic around the ring) + coupling
    nr = num.nr
    for k in range(spec.nz - 1):
        eta = spec.eta[k] if len(spec.eta) > 1 else spec.eta[0]
        for r in range(nr):
            r2 = (r + 1) % nr
            (i1, j1), (i2, j2) = num.ring[r], num.ring[r2]
            P1, P2 = xyz(i1, j1, k), xyz(i2, j2, k)
            L = np.linalg.norm(P2 - P1)
            X2 = np.array([[0.0, 0.0], [L, 0.0], [L, hz], [0.0, hz]])
            Ke, Me = cached('plate', X2, lambda X: mitc4_plate(X, spec.E, spec.nu, spec.rho_s, spec.t))
            sn = [(r, k), (r2, k), (r2, k + 1), (r, k + 1)]
            sd = [num.s(rr, kk, c) for (rr, kk) in sn for c in range(3)]
            put(Kr, Kc, Kv, sd, sd, Ke * (1.0 + 1j * eta))
            put(Mr, Mc, Mv, sd, sd, Me)
            # coupling through the wall face shared with the cavity
            fnodes = [(i1, j1, k), (i2, j2, k), (i2, j2, k + 1), (i1, j1, k + 1)]
            Xf = np.array([xyz(*nd) for nd in fnodes])
            Cf = cached('face', Xf, quad4_surface_mass)
            wd = [num.s(rr, kk, 0) for (rr, kk) in sn]
            pd = [num.p(*nd) for nd in fnodes]
            put(Kr, Kc, Kv, wd, pd, -Cf.astype(complex))         # K_sf = -C
            put(Mr, Mc, Mv, pd, wd, spec.rho * Cf.T)             # M_fs = rho C^T

    # ---- floor impedance on y = 0
    if spec.Z_floor is not None:
        beta = spec.rho / spec.Z_floor
        for k in range(spec.nz - 1):
            for i in range(spec.nx - 1):
                fnodes = [(i, 0, k), (i + 1, 0, k), (i + 1, 0, k + 1), (i, 0, k + 1)]
                Xf = np.array([xyz(*nd) for nd in fnodes])
                Mf = cached('face', Xf, quad4_surface_mass)
                pd = [num.p(*nd) for nd in fnodes]
                put(Dr, Dc, Dv, pd, pd, beta * Mf)

    n = num.n

    def build(R, Cc, V, dtype):
        if not R:
            return sp.csr_matrix((n, n), dtype=dtype)
        return sp.coo_matrix((np.concatenate(V).astype(dtype),
                              (np.concatenate(R), np.concatenate(Cc))), shape=(n, n)).tocsr()

    K = build(Kr, Kc, Kv, complex)
    M = build(Mr, Mc, Mv, float)
    D = build(Dr, Dc, Dv, complex)

    # ---- simply supported shell ends: w = 0 on slabs 0 and nz-1.  Rows and
    # columns are cleared, the stiffness diagonal is kept so A stays regular.
    fixed = np.array([num.s(r, k, 0) for k in (0, spec.nz - 1) for r in range(nr)])
    keep = np.ones(n)
    keep[fixed] = 0.0
    Pk = sp.diags(keep)
    kdiag = K.diagonal()
    fixdiag = np.zeros(n, dtype=complex)
    fixdiag[fixed] = kdiag[fixed]
    K = (Pk @ K @ Pk + sp.diags(fixdiag)).tocsr()
    M = (Pk @ M @ Pk).tocsr()
    D = (Pk @ D @ Pk).tocsr()
    for A_ in (K, M, D):
        A_.eliminate_zeros()
    is_fluid = np.zeros(n, dtype=bool)
    for k in range(spec.nz):
        is_fluid[k * num.b:k * num.b + num.npl] = True
    return Assembled(spec=spec, K=K, M=M, D=D, b=num.b, nz=spec.nz, n=n, is_fluid=is_fluid)


def load_matrix(spec, loads, n_rhs) -> np.ndarray:
    """Load vectors F (n x n_rhs): unit normal point forces on shell w-DoFs."""
    num = Numbering(spec)
    F = np.zeros((num.n, n_rhs), dtype=complex)
    for ld in loads:
        F[num.s(ld.ring, ld.slab, 0), ld.column] += ld.value
    return F


def receiver_dofs(spec, receivers) -> np.ndarray:
    num = Numbering(spec)
    return np.array([num.p(i, j, k) for (i, j, k) in receivers], dtype=np.int64)


def plate_mesh(a: float, c: float, nex: int, ney: int, E, nu, rho, t, eta=0.0):
    """Stand-alone rectangular plate [0,a] x [0,c] on nex x ney MITC4 elements.

    Returns (K, M, node_xy) with DoF 3*node + (w, beta_s, beta_z) and node =
    i + (nex+1)*j.  Used to pin the plate element against closed-form modes.
    """
    nnx, nny = nex + 1, ney + 1
    nn = nnx * nny
    K = np.zeros((3 * nn, 3 * nn), dtype=complex)
    M = np.zeros((3 * nn, 3 * nn))
    dx, dy = a / nex, c / ney
    for j in range(ney):
        for i in range(nex):
            nodes = [i + nnx * j, i + 1 + nnx * j, i + 1 + nnx * (j + 1), i + nnx * (j + 1)]
            X2 = np.array([[i * dx, j * dy], [(i + 1) * dx, j * dy],
                           [(i + 1) * dx, (j + 1) * dy], [i * dx, (j + 1) * dy]])
            Ke, Me = mitc4_plate(X2, E, nu, rho, t)
            d = [3 * nd + c_ for nd in nodes for c_ in range(3)]
            K[np.ix_(d, d)] += Ke * (1 + 1j * eta)
            M[np.ix_(d, d)] += Me
    xy = np.array([[i * dx, j * dy] for j in range(nny) for i in range(nnx)])
    return K, M, xy
