"""Pins for the oracle's FE assembly against closed forms and invariants.

Paper: Sec. 2 (problem statement, Eq. 1-3), Eq. 5 (coupling matrix), Sec. 3.3
(complex stiffness damping after Eq. 8).
"""
import numpy as np
import pytest
import scipy.linalg as la

import workloads as W
from oracle import fem


def _fluid_block(asm, spec):
    num = fem.Numbering(spec)
    idx = np.array([num.p(i, j, k) for k in range(spec.nz) for j in range(spec.ny)
                    for i in range(spec.nx)])
    I, J, K = np.meshgrid(np.arange(spec.nx), np.arange(spec.ny), np.arange(spec.nz), indexing="ij")
    I, J, K = (a.transpose(2, 1, 0).ravel() for a in (I, J, K))
    Kf = asm.K[idx][:, idx].toarray().real
    Mf = asm.M[idx][:, idx].toarray()
    return Kf, Mf, I, J, K


def _lam1d(l, N, h):
    th = l * np.pi / (N - 1)
    return 6.0 / h ** 2 * (1.0 - np.cos(th)) / (2.0 + np.cos(th))


@pytest.mark.parametrize("lmn", [(1, 0, 0), (0, 2, 1), (2, 1, 3), (3, 3, 2)])
def test_cavity_discrete_mode_exact(lmn):
    """cos-modes sampled at the nodes are exact generalised eigenvectors of the
    trilinear cavity with eigenvalue c^2 (lam_l + lam_m + lam_n)/c^2 (closed form)."""
    w = W.small_model(nx=5, ny=4, nz=6, floor=False)
    s = w.model
    asm = fem.assemble(s)
    Kf, Mf, I, J, K = _fluid_block(asm, s)
    l, m, n = lmn
    v = (np.cos(l * np.pi * I / (s.nx - 1)) * np.cos(m * np.pi * J / (s.ny - 1))
         * np.cos(n * np.pi * K / (s.nz - 1)))
    lam = (_lam1d(l, s.nx, s.Lx / (s.nx - 1)) + _lam1d(m, s.ny, s.Ly / (s.ny - 1))
           + _lam1d(n, s.nz, s.Lz / (s.nz - 1)))
    r = Kf @ v - lam * s.c ** 2 * (Mf @ v)
    assert np.linalg.norm(r) <= 1e-13 * max(np.linalg.norm(Kf @ v), 1.0)


def test_cavity_eigenfrequencies_converge_second_order():
    """Lowest rigid-wall cavity modes converge to c/2 sqrt((l/Lx)^2+(m/Ly)^2+(n/Lz)^2) at O(h^2)."""
    Lx, Ly, Lz, c = 0.6, 0.5, 1.0, 343.0
    exact = sorted(c / 2 * np.sqrt((l / Lx) ** 2 + (m / Ly) ** 2 + (n / Lz) ** 2)
                   for l in range(4) for m in range(4) for n in range(6))[1:6]
    errs = []
    for ref in (1, 2):
        w = W.small_model(nx=3 * ref + 1, ny=3 * ref + 1, nz=5 * ref + 1, Lx=Lx, Ly=Ly, Lz=Lz,
                          floor=False)
        asm = fem.assemble(w.model)
        Kf, Mf, *_ = _fluid_block(asm, w.model)
        ev = la.eigh(Kf, Mf, eigvals_only=True)
        f = np.sqrt(np.abs(ev[1:6])) / (2 * np.pi)
        errs.append(np.max(np.abs(f - exact) / exact))
    assert errs[1] < 0.06
    assert errs[0] / errs[1] > 3.2          # second order: ~4x per halving of h


def test_mass_and_coupling_sums():
    """sum(Mf) = V/c^2; each wall coupling block sums to the lined wall area;
    the floor damping sums to (rho/Z) * floor area; shell w-mass sums to rho_s t A."""
    w = W.small_model(nx=5, ny=4, nz=6)
    s = w.model
    asm = fem.assemble(s)
    fl = asm.is_fluid
    V = s.Lx * s.Ly * s.Lz
    assert np.isclose(asm.M[fl][:, fl].sum(), V / s.c ** 2, rtol=1e-13)
    num = fem.Numbering(s)
    wdofs = np.array([num.s(r, k, 0) for k in range(s.nz) for r in range(num.nr)])
    inner = np.array([num.s(r, k, 0) for k in range(1, s.nz - 1) for r in range(num.nr)])
    lateral = 2 * (s.Lx + s.Ly) * s.Lz
    # -K_sf summed over all w rows = C summed = lateral area (before the end BC removes rows)
    Csum_inner = -asm.K[inner][:, fl].sum().real
    Mfs = asm.M[fl][:, wdofs].sum() / s.rho
    hz = s.Lz / (s.nz - 1)
    # the two end slabs lose their w rows to the simply supported edge; their area share
    # is half an element height each
    assert np.isclose(Csum_inner, lateral - 2 * (2 * (s.Lx + s.Ly)) * hz / 2, rtol=1e-12)
    assert np.isclose(Mfs, lateral - 2 * (2 * (s.Lx + s.Ly)) * hz / 2, rtol=1e-12)
    Dsum = asm.D.sum()
    assert np.isclose(Dsum, s.rho / s.Z_floor * s.Lx * s.Lz, rtol=1e-12)
    # shell translational mass restricted to the w DoFs of the inner slabs: full
    # layers contribute rho_s t P hz, the two end layers rho_s t P hz/3 (one node of
    # the 1-D consistent mass (hz/6)[[2,1],[1,2]]).
    Mww = asm.M[inner][:, inner].sum()
    P = 2 * (s.Lx + s.Ly)
    assert np.isclose(Mww, s.rho_s * s.t * P * (s.Lz - 4 * hz / 3), rtol=1e-12)


def test_hex_element_rigid_and_linear_patch():
    """Ke annihilates constants; for a linear field the interior nodal flux vanishes."""
    X = np.array([[0, 0, 0], [0.3, 0, 0], [0.3, 0.2, 0], [0, 0.2, 0],
                  [0, 0, 0.4], [0.3, 0, 0.4], [0.3, 0.2, 0.4], [0, 0.2, 0.4]], dtype=float)
    Ke, Me = fem.hex8_matrices(X)
    assert np.abs(Ke @ np.ones(8)).max() < 1e-14
    assert np.isclose(Me.sum(), 0.3 * 0.2 * 0.4, rtol=1e-14)
    g = np.array([0.7, -1.3, 2.1])
    u = X @ g
    # energy of a linear field = |g|^2 * volume
    assert np.isclose(u @ Ke @ u, g @ g * 0.3 * 0.2 * 0.4, rtol=1e-13)


def _plate_ss_freqs(a, b, nex, ney, n_modes=4):
    s = W.ModelSpec(Lx=1, Ly=1, Lz=1, nx=2, ny=2, nz=2)
    K, M, xy = fem.plate_mesh(a, b, nex, ney, s.E, s.nu, s.rho_s, s.t)
    on_edge = (np.isclose(xy[:, 0], 0) | np.isclose(xy[:, 0], a) | np.isclose(xy[:, 1], 0)
               | np.isclose(xy[:, 1], b))
    fixed = 3 * np.where(on_edge)[0]
    free = np.setdiff1d(np.arange(K.shape[0]), fixed)
    ev = la.eigh(K[np.ix_(free, free)].real, M[np.ix_(free, free)], eigvals_only=True,
                 subset_by_index=[0, n_modes - 1])
    return np.sqrt(ev) / (2 * np.pi), s


def test_plate_simply_supported_modes_converge():
    """Simply supported rectangular plate: f_mn -> (pi/2)((m/a)^2+(n/b)^2) sqrt(D/(rho t))
    (Kirchhoff limit; t/a = 1/300 so transverse shear and rotary inertia are tiny)."""
    a, b = 0.6, 0.45
    errs = []
    for ne in (16, 32):
        f, s = _plate_ss_freqs(a, b, ne, int(ne * 3 / 4))
        Dp = s.E * s.t ** 3 / (12 * (1 - s.nu ** 2))
        exact = sorted(np.pi / 2 * ((m / a) ** 2 + (n / b) ** 2) * np.sqrt(Dp / (s.rho_s * s.t))
                       for m in range(1, 5) for n in range(1, 5))[:4]
        errs.append(np.max(np.abs(f - exact) / exact))
    assert errs[1] < 0.01
    assert errs[0] > 3.5 * errs[1]          # O(h^2): no shear locking at t/a = 1/300


def test_developed_ring_plate_modes():
    """The shell ring alone (periodic in s, simply supported ends) has modes
    f = (1/2pi) sqrt(D/(rho t)) [(m pi/L)^2 + (2 pi n/P)^2] with P the perimeter."""
    w = W.small_model(nx=9, ny=9, nz=13, Lx=0.5, Ly=0.5, Lz=0.8, floor=False, eta=0.0)
    s = w.model
    asm = fem.assemble(s)
    sh = ~asm.is_fluid
    num = fem.Numbering(s)
    fixed = set(num.s(r, k, 0) for k in (0, s.nz - 1) for r in range(num.nr))
    idx = np.array([i for i in np.where(sh)[0] if i not in fixed])
    K = asm.K[idx][:, idx].toarray().real
    M = asm.M[idx][:, idx].toarray()
    ev = la.eigh(K, M, eigvals_only=True, subset_by_index=[0, 5])
    f = np.sqrt(ev) / (2 * np.pi)
    Dp = s.E * s.t ** 3 / (12 * (1 - s.nu ** 2))
    P = 2 * (s.Lx + s.Ly)
    ex = sorted(np.sqrt(Dp / (s.rho_s * s.t)) / (2 * np.pi) * ((m * np.pi / s.Lz) ** 2 +
                (2 * np.pi * n / P) ** 2) for m in range(1, 4) for n in range(0, 4)
                for _ in ((0,) if n == 0 else (0, 1)))[:6]
    assert np.max(np.abs(f - ex) / ex) < 0.05


def test_damping_enters_as_complex_stiffness():
    """Shell stiffness carries (1 + i eta); the fluid block is real (Sec. 3.3)."""
    w = W.small_model(eta=0.02, floor=False)
    asm = fem.assemble(w.model)
    sh = ~asm.is_fluid
    Ks = asm.K[sh][:, sh].toarray()
    ratio = Ks.imag[np.abs(Ks.real) > 1e-6 * np.abs(Ks.real).max()] / Ks.real[np.abs(Ks.real) > 1e-6 * np.abs(Ks.real).max()]
    # every off-diagonal and non-BC diagonal entry has imag/real = eta
    assert np.allclose(ratio[np.abs(ratio) > 0], 0.02, rtol=1e-12)
    fl = asm.is_fluid
    assert np.abs(asm.K[fl][:, fl].toarray().imag).max() == 0.0


def test_element_shape_functions_and_matrices_closed_forms():
    """Element-level pins: trilinear / bilinear shape functions interpolate the nodes and
    sum to one; the unit-cube Laplacian and mass have the textbook diagonal 1/3 and 1/27
    and sum to 0 and the volume; the surface mass of a tilted rectangle sums to its area
    with diagonal area/9 and opposite-corner entry area/36."""
    rng = np.random.default_rng(0)
    for a, node in enumerate(fem.HEX_NODES):
        N, _ = fem.hex8_shape(*node)
        assert np.allclose(N, np.eye(8)[a])
    for _ in range(5):
        N, dN = fem.hex8_shape(*rng.uniform(-1, 1, 3))
        assert N.sum() == pytest.approx(1.0) and np.allclose(dN.sum(axis=0), 0.0)
        N, dN = fem.quad4_shape(*rng.uniform(-1, 1, 2))
        assert N.sum() == pytest.approx(1.0) and np.allclose(dN.sum(axis=0), 0.0)
    X = (fem.HEX_NODES + 1.0) / 2.0                       # unit cube
    Ke, Me = fem.hex8_matrices(X)
    assert np.allclose(np.diag(Ke), 1.0 / 3.0) and np.allclose(Ke @ np.ones(8), 0.0)
    assert np.allclose(np.diag(Me), 1.0 / 27.0) and Me.sum() == pytest.approx(1.0)
    Xb = X * np.array([0.5, 2.0, 3.0])                    # box: Laplacian scales, mass sums to the volume
    Ke_b, Me_b = fem.hex8_matrices(Xb)
    assert Me_b.sum() == pytest.approx(3.0) and np.allclose(Ke_b @ np.ones(8), 0.0)
    a, b = 0.7, 1.9
    R = la.expm(np.array([[0, -0.3, 0.2], [0.3, 0, -0.5], [-0.2, 0.5, 0]]))   # a rotation
    Xq = np.array([[0, 0, 0], [a, 0, 0], [a, b, 0], [0, b, 0]], dtype=float) @ R.T + 1.5
    Mq = fem.quad4_surface_mass(Xq)
    assert Mq.sum() == pytest.approx(a * b)
    assert np.allclose(np.diag(Mq), a * b / 9.0) and Mq[0, 2] == pytest.approx(a * b / 36.0)


def test_mitc4_plate_rigid_modes_and_mass():
    """The Reissner-Mindlin element (shear strain grad w + beta) stores no energy in the
    three rigid modes of a plate: translation w = 1, and rotations w = s with beta_s = -1,
    w = z with beta_z = -1; its translational mass is rho t times the area; a pure bending
    field (w = s^2 / 2, beta_s = -s) is not rigid."""
    X2 = np.array([[0.0, 0.0], [0.8, 0.1], [0.9, 1.1], [-0.1, 0.9]])
    Ke, Me = fem.mitc4_plate(X2, 60e9, 0.3, 1600.0, 0.002)
    assert np.allclose(Ke, Ke.T, rtol=1e-12, atol=1e-9 * np.abs(Ke).max())
    modes = []
    u = np.zeros(12); u[0::3] = 1.0; modes.append(u)
    u = np.zeros(12); u[0::3] = X2[:, 0]; u[1::3] = -1.0; modes.append(u)
    u = np.zeros(12); u[0::3] = X2[:, 1]; u[2::3] = -1.0; modes.append(u)
    scale = np.abs(Ke).max()
    for u in modes:
        assert np.abs(Ke @ u).max() < 1e-9 * scale
    d1, d2 = X2[2] - X2[0], X2[3] - X2[1]
    area = 0.5 * abs(d1[0] * d2[1] - d1[1] * d2[0])
    w = np.zeros(12); w[0::3] = 1.0
    assert w @ Me @ w == pytest.approx(1600.0 * 0.002 * area, rel=1e-12)
    u = np.zeros(12); u[0::3] = X2[:, 0] ** 2 / 2.0; u[1::3] = -X2[:, 0]
    assert u @ Ke @ u > 1e-6 * scale


def test_ring_nodes_walk_the_perimeter_counter_clockwise():
    for nx, ny in ((3, 4), (8, 8), (24, 24)):
        ring = fem.ring_nodes(nx, ny)
        assert len(ring) == 2 * nx + 2 * ny - 4 == len(set(ring))
        assert ring[0] == (0, 0) and ring[1] == (1, 0) and ring[-1] == (0, 1)
        assert all(i in (0, nx - 1) or j in (0, ny - 1) for i, j in ring)
        steps = [abs(a[0] - b[0]) + abs(a[1] - b[1]) for a, b in zip(ring, ring[1:] + ring[:1])]
        assert steps == [1] * len(ring)


# --------------------------------------------------------------------------- floor impedance
def _floor_pressure_energy(spec, p_nodes):
    """int_floor |p|^2 dGamma of the bilinear interpolant of nodal pressures on y = 0, by
    the closed form of the bilinear element's mass on an hx x hz rectangle
    (hx hz / 36) [4 2 1 2; 2 4 2 1; 1 2 4 2; 2 1 2 4], written out here independently of the
    oracle's quadrature."""
    hx = spec.Lx / (spec.nx - 1)
    hz = spec.Lz / (spec.nz - 1)
    Me = hx * hz / 36.0 * np.array([[4, 2, 1, 2], [2, 4, 2, 1], [1, 2, 4, 2], [2, 1, 2, 4]], float)
    tot = 0.0
    for k in range(spec.nz - 1):
        for i in range(spec.nx - 1):
            v = np.array([p_nodes[i, k], p_nodes[i + 1, k], p_nodes[i + 1, k + 1], p_nodes[i, k + 1]])
            tot += float(np.real(np.conj(v) @ Me @ v))
    return tot


def _power_balance(asm, spec, w, freq, flip_damping=False):
    """Time-averaged power injected by the unit shell force and absorbed by the floor."""
    num = fem.Numbering(spec)
    om = 2 * np.pi * freq
    A = (asm.K + (-1j if flip_damping else 1j) * om * asm.D - om ** 2 * asm.M).tocsc()
    F = fem.load_matrix(spec, w.loads, w.n_rhs)[:, 0]
    import scipy.sparse.linalg as spla
    x = spla.spsolve(A, F)
    a = np.flatnonzero(F)[0]
    # e^{+i w t}: shell velocity i w x_a; P_in = 1/2 Re(conj(v_a) F_a)
    p_in = 0.5 * np.real(np.conj(1j * om * x[a]) * F[a])
    p_floor_nodes = np.array([[x[num.p(i, 0, k)] for k in range(spec.nz)] for i in range(spec.nx)])
    # locally reacting wall: normal velocity into the wall v_n = p / Z, P = 1/2 Re(p conj(v_n))
    p_floor = 0.5 * np.real(1.0 / np.conj(spec.Z_floor)) * _floor_pressure_energy(spec, p_floor_nodes)
    return p_in, p_floor


def test_power_balance_of_the_floor_impedance():
    """With the shell undamped (eta = 0) the floor impedance (Re Z > 0) is the only loss: the
    power the point force injects, 1/2 Re(conj(i w w_a) F_a), equals the power the floor
    absorbs, 1/2 Re(1/Z) int_floor |p|^2, and is positive (paper Sec. 2 problem statement,
    Eq. 8 damping term).  The identity holds exactly for the discrete system (the shell's and
    cavity's stiffness and mass forms are real symmetric and the coupling enters the shell and
    fluid rows with the signs of the weak form), so any slip in the sign of i w D, in the sign
    of the coupling or in rho/Z breaks it.  A flipped damping term is planted to show it."""
    spec = W.ModelSpec(Lx=0.6, Ly=0.5, Lz=0.8, nx=5, ny=4, nz=6, eta=(0.0,),
                       Z_floor=W.AIR_RHO * W.AIR_C * (1.5 - 0.7j))
    w = W.Workload(name="power-balance", config_id=91, model=spec,
                                  loads=(W.PointLoad(slab=2, ring=3, column=0),), n_rhs=1, receivers=((1, 1, 1),),
                                  freqs_hz=np.array([1.0]))
    asm = fem.assemble(spec)
    for f in (61.0, 143.0, 377.0):
        p_in, p_floor = _power_balance(asm, spec, w, f)
        assert p_in > 0.0
        assert abs(p_in - p_floor) <= 1e-9 * p_in, (f, p_in, p_floor)
        bad_in, bad_floor = _power_balance(asm, spec, w, f, flip_damping=True)
        assert bad_in < 0.0 and abs(bad_in - bad_floor) > 0.5 * abs(bad_floor)


def test_impedance_tube_closed_form():
    """The cavity block alone (rigid side walls, no shell) driven by a uniform normal pressure
    gradient g on the face y = Ly, with the locally reacting impedance Z on y = 0, is a 1-D
    problem: p(y) = a cos(ky) + b sin(ky), p'(0) = i k (rho c / Z) p(0) (the floor condition
    dp/dn = -i w rho p / Z, n = -y), p'(Ly) = g.  The trilinear solution converges to it at
    O(h^2); the reactive part of Z enters the phase, so a conjugated Z (rho / conj(Z)) or a
    flipped damping sign misses it by orders of magnitude."""
    import scipy.sparse.linalg as spla
    Z = W.AIR_RHO * W.AIR_C * (0.8 + 1.3j)
    f, g, Ly = 150.0, 1.0, 1.0
    om = 2 * np.pi * f
    k = om / W.AIR_C
    a = g / (k * (-np.sin(k * Ly) + 1j * (W.AIR_RHO * W.AIR_C / Z) * np.cos(k * Ly)))
    b = 1j * (W.AIR_RHO * W.AIR_C / Z) * a

    def exact(y):
        return a * np.cos(k * y) + b * np.sin(k * y)

    def solve(ny, variant=None):
        spec = W.ModelSpec(Lx=0.3, Ly=Ly, Lz=0.4, nx=3, ny=ny, nz=3, eta=(0.0,), Z_floor=Z)
        asm = fem.assemble(spec)
        fl = np.flatnonzero(asm.is_fluid)
        D = asm.D[fl][:, fl]
        if variant == "conj":
            D = D.conj()
        sgn = -1j if variant == "flip" else 1j
        A = (asm.K[fl][:, fl] + sgn * om * D - om ** 2 * asm.M[fl][:, fl]).tocsc()
        num = fem.Numbering(spec)
        # consistent load of a uniform g on the top face: g times the nodal tributary areas
        hx, hz = spec.Lx / (spec.nx - 1), spec.Lz / (spec.nz - 1)
        rhs = np.zeros(spec.n, complex)
        for kk in range(spec.nz):
            for i in range(spec.nx):
                wx = 0.5 if i in (0, spec.nx - 1) else 1.0
                wz = 0.5 if kk in (0, spec.nz - 1) else 1.0
                rhs[num.p(i, ny - 1, kk)] = g * hx * hz * wx * wz
        p = spla.spsolve(A, rhs[fl])
        full = np.zeros(spec.n, complex)
        full[fl] = p
        ys = np.linspace(0.0, Ly, ny)
        got = np.array([full[num.p(1, j, 1)] for j in range(ny)])
        return np.abs(got - exact(ys)).max() / np.abs(exact(ys)).max()

    e1, e2 = solve(33), solve(65)
    print("impedance tube errors", e1, e2)
    assert e2 < 1e-3 and 3.0 < e1 / e2 < 5.0        # O(h^2)
    assert solve(65, "conj") > 100 * e2
    assert solve(65, "flip") > 100 * e2
