"""Seeded synthetic workloads for the coupled shell-cavity frequency sweep.

This module is shared by the oracle (``oracle/``) and the CUDA path
(``paper_2310_04734_gb300``).  It holds only the *inputs*: geometry, material
constants, the random draws (load positions, receiver nodes, per-layer loss
factors, check frequencies, design variants) and the frequency grids.  It
contains none of the method's arithmetic (no element matrices, no solves), and
imports nothing from either side.

Every random draw comes from ``numpy.random.default_rng([config_id, stream])``
with one stream per kind of draw:

    stream 0  load positions        stream 3  check frequencies
    stream 1  receiver nodes        stream 4  design variants
    stream 2  loss factor per layer stream 5  estimator initialisation

The model follows the paper's problem statement (Sec. 2, Eq. 1-3): a
rectangular air cavity meshed with trilinear pressure elements whose four
lateral walls are lined by a Reissner-Mindlin shell ring, coupled through the
wall-normal displacement; structural damping enters as a complex stiffness
K(1 + i eta) (Sec. 3.3, text after Eq. 8); a locally reacting floor impedance adds a
damping matrix D.  The slab-major DoF ordering (slab k = nodes with z-index
k: first the nx*ny pressure DoFs, then 3 DoFs per shell ring node) is the
convention both sides use to index loads and receivers.
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace
from typing import List, Optional, Tuple

import numpy as np

AIR_C = 343.0          # speed of sound, m/s
AIR_RHO = 1.21         # air density, kg/m^3
SHELL_E = 60e9         # Young's modulus, Pa
SHELL_NU = 0.3
SHELL_RHO = 1600.0     # kg/m^3
SHELL_T = 2e-3         # m
P_REF = 2e-5           # Pa, SPL reference pressure


@dataclass(frozen=True)
class ModelSpec:
    """Geometry and materials of one coupled shell-cavity model."""
    Lx: float
    Ly: float
    Lz: float
    nx: int
    ny: int
    nz: int
    c: float = AIR_C
    rho: float = AIR_RHO
    E: float = SHELL_E
    nu: float = SHELL_NU
    rho_s: float = SHELL_RHO
    t: float = SHELL_T
    # loss factor of each shell element layer between slabs k and k+1 (nz-1 values)
    eta: Tuple[float, ...] = ()
    # locally reacting impedance on the floor face y = 0 (None: rigid floor)
    Z_floor: Optional[complex] = None

    @property
    def n_ring(self) -> int:
        return 2 * (self.nx - 1) + 2 * (self.ny - 1)

    @property
    def n_press_slab(self) -> int:
        return self.nx * self.ny

    @property
    def b(self) -> int:
        return self.n_press_slab + 3 * self.n_ring

    @property
    def n(self) -> int:
        return self.b * self.nz


@dataclass(frozen=True)
class PointLoad:
    """Unit normal point force on the shell: w-DoF of ring node ``ring`` of slab ``slab``."""
    slab: int
    ring: int
    column: int
    value: complex = 1.0 + 0.0j


@dataclass(frozen=True)
class Workload:
    name: str
    config_id: int
    model: ModelSpec
    loads: Tuple[PointLoad, ...]
    n_rhs: int
    receivers: Tuple[Tuple[int, int, int], ...]   # interior pressure nodes (i, j, k)
    freqs_hz: np.ndarray = field(compare=False)
    check_freqs_hz: Optional[np.ndarray] = field(default=None, compare=False)
    precision: str = "fp64"


def _rng(config_id: int, stream: int) -> np.random.Generator:
    return np.random.default_rng([config_id, stream])


def _receivers(cfg_id: int, nx: int, ny: int, nz: int, count: int):
    """``count`` distinct strictly interior pressure nodes, drawn without replacement."""
    rng = _rng(cfg_id, 1)
    ni, nj, nk = nx - 2, ny - 2, nz - 2
    flat = rng.choice(ni * nj * nk, size=count, replace=False)
    out = []
    for f in flat:
        f = int(f)
        i = f % ni
        j = (f // ni) % nj
        k = f // (ni * nj)
        out.append((i + 1, j + 1, k + 1))
    return tuple(out)


def _shell_loads(cfg_id: int, nz: int, n_ring: int, count: int):
    """``count`` unit shell point forces at seeded (slab, ring) positions, one per column.

    Slabs 0 and nz-1 carry the simply supported shell edges (w = 0), so loads are
    drawn from slabs 1..nz-2.
    """
    rng = _rng(cfg_id, 0)
    seen = set()
    loads = []
    col = 0
    while len(loads) < count:
        slab = int(rng.integers(1, nz - 1))
        ring = int(rng.integers(0, n_ring))
        if (slab, ring) in seen:
            continue
        seen.add((slab, ring))
        loads.append(PointLoad(slab=slab, ring=ring, column=col))
        col += 1
    return tuple(loads)


def config1() -> Workload:
    """Tiny plain FP64 sweep: 1x1x2 m cavity, 8x8x16 nodes, 181 frequencies."""
    m = ModelSpec(Lx=1.0, Ly=1.0, Lz=2.0, nx=8, ny=8, nz=16, eta=(0.01,) * 15)
    loads = (PointLoad(slab=8, ring=3, column=0),)
    return Workload(name="cfg1_tiny_fp64", config_id=1, model=m, loads=loads, n_rhs=1,
                    receivers=_receivers(1, m.nx, m.ny, m.nz, 8),
                    freqs_hz=np.arange(20.0, 200.0 + 0.5, 1.0))


def config2() -> Workload:
    """Medium plain FP64 sweep: 1.5x1.5x6 m cavity, 24x24x96 nodes, floor impedance,
    4 seeded shell loads, 32 receivers, 481 frequencies (20-500 Hz)."""
    m = ModelSpec(Lx=1.5, Ly=1.5, Lz=6.0, nx=24, ny=24, nz=96, eta=(0.01,) * 95,
                  Z_floor=AIR_RHO * AIR_C * (2.0 - 1.0j))
    return Workload(name="cfg2_medium_fp64", config_id=2, model=m,
                    loads=_shell_loads(2, m.nz, m.n_ring, 4), n_rhs=4,
                    receivers=_receivers(2, m.nx, m.ny, m.nz, 32),
                    freqs_hz=np.arange(20.0, 500.0 + 0.5, 1.0))


def config3() -> Workload:
    """Mixed precision on the config-1 model (same model, loads, receivers, grid)."""
    w = config1()
    return replace(w, name="cfg3_tiny_mixed", config_id=3, precision="mixed")


def config4() -> Workload:
    """Rational Arnoldi MOR: 2x2x10 m cavity, 32x32x160 nodes, eta per layer
    U[0.005, 0.03], 2 loads, 64 receivers, 2000 frequencies on a 0.5 Hz grid,
    50 seeded check frequencies."""
    eta = _rng(4, 2).uniform(0.005, 0.03, size=159)
    m = ModelSpec(Lx=2.0, Ly=2.0, Lz=10.0, nx=32, ny=32, nz=160, eta=tuple(float(e) for e in eta))
    freqs = 0.5 * np.arange(1, 2001, dtype=np.float64)
    chk = np.sort(_rng(4, 3).choice(freqs, size=50, replace=False))
    return Workload(name="cfg4_rom", config_id=4, model=m,
                    loads=_shell_loads(4, m.nz, m.n_ring, 2), n_rhs=2,
                    receivers=_receivers(4, m.nx, m.ny, m.nz, 64),
                    freqs_hz=freqs, check_freqs_hz=chk)


def config5_variants(count: int = 64) -> List[Workload]:
    """Design-study variants: nz U{96..200}, cross-section 24x24 (1.5x1.5 m) or 32x32
    (2x2 m), t U[1.5, 3] mm, floor impedance rho*c*(a - 1i) with a U[1, 4]; one
    seeded load and 32 receivers each; 1600 frequencies on a 0.5 Hz grid."""
    rng = _rng(5, 4)
    out = []
    freqs = 0.5 * np.arange(1, 1601, dtype=np.float64)
    for v in range(count):
        nz = int(rng.integers(96, 201))
        big = bool(rng.integers(0, 2))
        t = float(rng.uniform(1.5e-3, 3e-3))
        a = float(rng.uniform(1.0, 4.0))
        nxy = 32 if big else 24
        L = 2.0 if big else 1.5
        m = ModelSpec(Lx=L, Ly=L, Lz=(nz - 1) * 6.0 / 95.0, nx=nxy, ny=nxy, nz=nz, t=t,
                      eta=(0.01,) * (nz - 1), Z_floor=AIR_RHO * AIR_C * (a - 1.0j))
        cid = 1000 + v
        out.append(Workload(name=f"cfg5_variant{v:02d}", config_id=cid, model=m,
                            loads=_shell_loads(cid, nz, m.n_ring, 1), n_rhs=1,
                            receivers=_receivers(cid, nxy, nxy, nz, 32), freqs_hz=freqs))
    return out


def config5_reduced_variants(count: int = 64) -> List[Workload]:
    """Config 5's design study at a scale one GPU runs in minutes: the same variant
    recipe (seeded nz, two cross-sections, shell thickness U[1.5, 3] mm, floor
    impedance rho*c*(a - 1i), a U[1, 4]; one load) on coarse meshes -- nz U{10..20}
    slabs of 6 x 6 (0.6 x 0.6 m) or 8 x 8 (0.8 x 0.8 m) nodes, axial spacing 0.1 m --
    8 receivers, 101 frequencies on a 1 Hz grid over 20-120 Hz (the band a ROM of
    about a hundred columns resolves for shells this thin)."""
    rng = _rng(5, 7)
    out = []
    freqs = 20.0 + 1.0 * np.arange(101, dtype=np.float64)
    for v in range(count):
        nz = int(rng.integers(10, 21))
        big = bool(rng.integers(0, 2))
        t = float(rng.uniform(1.5e-3, 3e-3))
        a = float(rng.uniform(1.0, 4.0))
        nxy = 8 if big else 6
        L = 0.8 if big else 0.6
        m = ModelSpec(Lx=L, Ly=L, Lz=(nz - 1) * 0.1, nx=nxy, ny=nxy, nz=nz, t=t,
                      eta=(0.01,) * (nz - 1), Z_floor=AIR_RHO * AIR_C * (a - 1.0j))
        cid = 2000 + v
        out.append(Workload(name=f"cfg5r_variant{v:02d}", config_id=cid, model=m,
                            loads=_shell_loads(cid, nz, m.n_ring, 1), n_rhs=1,
                            receivers=_receivers(cid, nxy, nxy, nz, 8), freqs_hz=freqs))
    return out


def small_model(nx: int = 5, ny: int = 4, nz: int = 6, Lx: float = 0.6, Ly: float = 0.5,
                Lz: float = 1.0, floor: bool = True, eta: float = 0.02, t: float = SHELL_T,
                cfg_id: int = 99, n_loads: int = 2, n_rcv: int = 4) -> Workload:
    """A tiny, deliberately non-square model for brute-force checks (dense solves)."""
    m = ModelSpec(Lx=Lx, Ly=Ly, Lz=Lz, nx=nx, ny=ny, nz=nz, t=t, eta=(eta,) * (nz - 1),
                  Z_floor=(AIR_RHO * AIR_C * (2.0 - 1.0j)) if floor else None)
    return Workload(name=f"small_{nx}x{ny}x{nz}", config_id=cfg_id, model=m,
                    loads=_shell_loads(cfg_id, nz, m.n_ring, n_loads), n_rhs=n_loads,
                    receivers=_receivers(cfg_id, nx, ny, nz, n_rcv),
                    freqs_hz=np.linspace(30.0, 300.0, 10))


CONFIGS = {1: config1, 2: config2, 3: config3, 4: config4}


# ----------------------------------------------------------------- learned estimator
def mlp_init(stream: int = 5) -> np.ndarray:
    """Seeded initial parameters of the 5-64-64-1 error estimator, flat in the layout
    [W1 (64x5, row-major), b1, W2 (64x64), b2, W3 (1x64), b3]: Glorot-uniform
    weights, zero biases (config 5, stream 5)."""
    rng = _rng(5, stream)
    parts = []
    for fan_in, fan_out in ((5, 64), (64, 64), (64, 1)):
        lim = np.sqrt(6.0 / (fan_in + fan_out))
        parts.append(rng.uniform(-lim, lim, size=fan_out * fan_in))
        parts.append(np.zeros(fan_out))
    return np.concatenate(parts)


def mlp_order(n_samples: int, steps: int, batch: int, stream: int = 6) -> np.ndarray:
    """Seeded mini-batch rows (steps x batch, int32) for training on n_samples rows."""
    return _rng(5, stream).integers(0, n_samples, size=(steps, batch)).astype(np.int32)

