"""Seeded synthetic inputs for the phonon BTE hot path.

This module is shared by the CUDA path's callers (tests, bench) and by the CPU
oracle's callers.  It holds input recipes only -- geometries, band parameters,
wall temperatures, step counts -- and none of the method's arithmetic (no
direction sets, no quadrature, no equilibrium intensity, no update formula).

The paper (Sec. 3.1, "Model") discretises frequency into 40 bands, giving 55
band-polarisations (40 longitudinal + 15 transverse), uses 20x20 = 400
directions for 3-D problems and a 2-D test case with a hot-spot wall and an
opposite cold wall.  It prints no dispersion data, so the band parameters are
drawn from a seeded counter-based generator:

* frequency edges split [0, 1e14] rad/s evenly;
* group velocity v_b ~ U[1e3, 8e3] m/s, relaxation time tau_b = 10^U[-12,-9] s;
* longitudinal branch on every interval (degeneracy 1), transverse branch on
  the lowest ``n_ta`` intervals (degeneracy 2);
* draws: v for every band in band order, then tau, from SplitMix64.

SplitMix64 is the published generator of Steele, Lea and Flood (OOPSLA 2014);
a double in [0, 1) is its top 53 bits times 2^-53.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

MASK64 = (1 << 64) - 1

# Boundary-condition kinds and side numbering used by every caller.
BC_ISOTHERMAL = 0
BC_SPECULAR = 1
BC_DIFFUSE = 2   # fully diffuse wall: incoming intensity isotropic, carrying the outgoing energy flux
BC_PARTIAL = 3   # partially specular wall: (BC_PARTIAL, p) mixes p x mirror + (1 - p) x diffuse
SIDES = ("-x", "+x", "-y", "+y", "-z", "+z")


class SplitMix64:
    """SplitMix64 (Steele, Lea, Flood 2014): a 64-bit counter-based generator."""

    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)

    def uniform(self) -> float:
        """Top 53 bits times 2^-53: a double in [0, 1)."""
        return (self.next_u64() >> 11) * (1.0 / 9007199254740992.0)

    def randint(self, lo: int, hi: int) -> int:
        """Integer uniform on {lo..hi} (inclusive) by scaling one uniform draw."""
        return lo + int(self.uniform() * (hi - lo + 1))


@dataclass
class Bands:
    omega_lo: np.ndarray
    omega_hi: np.ndarray
    vg: np.ndarray
    beta: np.ndarray          # 1/tau, per band [1/s]
    degeneracy: np.ndarray

    @property
    def nb(self) -> int:
        return int(self.vg.shape[0])


def make_bands(n_intervals: int, n_ta: int, seed: int, omega_max: float = 1e14,
               v_range=(1e3, 8e3), log10_tau_range=(-12.0, -9.0)) -> Bands:
    """Band-polarisation table: LA on all intervals, then TA on the lowest n_ta."""
    edges = [omega_max * i / n_intervals for i in range(n_intervals + 1)]
    lo = [edges[i] for i in range(n_intervals)] + [edges[i] for i in range(n_ta)]
    hi = [edges[i + 1] for i in range(n_intervals)] + [edges[i + 1] for i in range(n_ta)]
    g = [1.0] * n_intervals + [2.0] * n_ta
    nb = n_intervals + n_ta
    rng = SplitMix64(seed)
    v = [v_range[0] + (v_range[1] - v_range[0]) * rng.uniform() for _ in range(nb)]
    tau = [10.0 ** (log10_tau_range[0] + (log10_tau_range[1] - log10_tau_range[0]) * rng.uniform())
           for _ in range(nb)]
    return Bands(np.array(lo), np.array(hi), np.array(v), 1.0 / np.array(tau), np.array(g))


@dataclass
class Geometry:
    dim: int
    nx: int
    ny: int
    nz: int
    dx: float
    dy: float
    dz: float
    # per side: (kind, per-face temperatures or None)
    bc: list = field(default_factory=list)
    T_init: float = 300.0

    @property
    def ncells(self) -> int:
        return self.nx * self.ny * self.nz

    def nfaces(self, side: int) -> int:
        """Faces on a side; face index along the wall as in the C headers."""
        if side < 2:
            return self.ny * self.nz
        if side < 4:
            return self.nx * self.nz
        return self.nx * self.ny


@dataclass
class Dirs:
    kind: str      # "inplane" or "polar_azim"
    n_inplane: int = 0
    n_polar: int = 0
    n_azim: int = 0

    @property
    def nd(self) -> int:
        return self.n_inplane if self.kind == "inplane" else self.n_polar * self.n_azim


@dataclass
class Workload:
    name: str
    geoms: list
    dirs: Dirs
    bands: Bands
    dt: float
    nsteps: int
    ninner: int
    precision: str = "fp64"

    @property
    def dof(self) -> int:
        return sum(g.ncells for g in self.geoms) * self.dirs.nd * self.bands.nb

    @property
    def updates(self) -> int:
        return self.dof * self.nsteps * self.ninner


def uniform_walls(geom: Geometry, kinds, temps):
    """Fill geom.bc from per-side kinds and uniform temperatures (None for
    specular and diffuse sides; for partially specular sides temps gives the
    specularity p)."""
    geom.bc = []
    nsides = 2 * geom.dim
    for s in range(nsides):
        if kinds[s] == BC_ISOTHERMAL:
            geom.bc.append((BC_ISOTHERMAL, np.full(geom.nfaces(s), float(temps[s]))))
        elif kinds[s] == BC_PARTIAL:
            geom.bc.append((BC_PARTIAL, float(temps[s])))
        else:
            geom.bc.append((BC_DIFFUSE if kinds[s] == BC_DIFFUSE else BC_SPECULAR, None))
    return geom


def hot_spot_profile(n: int, T_base: float, dT: float, r_cells: float) -> np.ndarray:
    """Gaussian wall-temperature profile: T_base + dT*exp(-2 (y - y_c)^2 / r^2), in cell units.

    The paper's hot spot (Sec. 3.1) is a centred Gaussian with a 1/e^2 half-width;
    the factor 2 makes r that 1/e^2 distance.
    """
    y = np.arange(n) + 0.5
    yc = n / 2.0
    return T_base + dT * np.exp(-2.0 * (y - yc) ** 2 / r_cells ** 2)


# ---------------------------------------------------------------------------
# The five workloads (sizes, seeds, walls).  Seeds are 19400 + workload number.
# ---------------------------------------------------------------------------


def paper_hot_spot(n: int = 120, nsteps: int = 100, ninner: int = 1) -> "Workload":
    """The paper's demonstration device (Sec. 3.1-3.2): a 2-D square of side
    525 um on an n x n grid (n = 120), 20 uniformly spaced in-plane directions,
    40 frequency bands giving 55 band-pols, initial equilibrium at 300 K.  The
    -x wall is isothermal with a centred Gaussian hot spot (350 K peak, 1/e^2
    distance 10 um), the +x wall is the 300 K cold wall, +-y are symmetric.
    Time step 1 ns (100 steps = 100 ns).  The band table comes from the
    synthetic generator (seed 19406): the paper gives no dispersion or
    relaxation-time data."""
    side = 525e-6
    d = side / n
    g = Geometry(2, n, n, 1, d, d, d)
    g.bc = [(BC_ISOTHERMAL, hot_spot_profile(n, 300.0, 50.0, 10e-6 / d)),
            (BC_ISOTHERMAL, np.full(n, 300.0)),
            (BC_SPECULAR, None), (BC_SPECULAR, None)]
    return Workload(f"paper_2d_{n}x{n}_20dir_55band_fp64", [g], Dirs("inplane", n_inplane=20),
                    make_bands(40, 15, 19406), 1e-9, nsteps, ninner, "fp64")

def cfg1() -> Workload:
    """2-D 20x20, 10 nm cells, 16 in-plane directions, 4 bands; -x wall 305 K, others 300 K."""
    g = Geometry(2, 20, 20, 1, 10e-9, 10e-9, 10e-9)
    uniform_walls(g, [BC_ISOTHERMAL] * 4, [305.0, 300.0, 300.0, 300.0])
    return Workload("2d_20x20_16dir_4band_fp64", [g], Dirs("inplane", n_inplane=16),
                    make_bands(4, 0, 19401), 1e-12, 100, 10, "fp64")


def cfg2(nx: int = 128, ny: int = 128, nsteps: int = 200, ninner: int = 15) -> Workload:
    """2-D 128x128, 400 directions (20 polar x 20 azimuthal), 55 band-pols, FP64.

    -x wall: Gaussian hot spot peaking near 310 K (r = 8 cells); +x wall 300 K;
    +-y walls specular.
    """
    g = Geometry(2, nx, ny, 1, 10e-9, 10e-9, 10e-9)
    g.bc = [(BC_ISOTHERMAL, hot_spot_profile(ny, 300.0, 10.0, 8.0)),
            (BC_ISOTHERMAL, np.full(ny, 300.0)),
            (BC_SPECULAR, None), (BC_SPECULAR, None)]
    return Workload(f"2d_{nx}x{ny}_400dir_55band_fp64", [g], Dirs("polar_azim", n_polar=20, n_azim=20),
                    make_bands(40, 15, 19402), 1e-12, nsteps, ninner, "fp64")


def cfg3(n: int = 64, precision: str = "fp32", nsteps: int = 100, ninner: int = 15) -> Workload:
    """3-D n^3, 400 directions, 55 band-pols; x walls 300/305 K, specular y and z."""
    g = Geometry(3, n, n, n, 10e-9, 10e-9, 10e-9)
    uniform_walls(g, [BC_ISOTHERMAL, BC_ISOTHERMAL] + [BC_SPECULAR] * 4, [300.0, 305.0, 0, 0, 0, 0])
    return Workload(f"3d_{n}^3_400dir_55band_{precision}", [g], Dirs("polar_azim", n_polar=20, n_azim=20),
                    make_bands(40, 15, 19403), 1e-12, nsteps, ninner, precision)


def cfg4(nx: int = 100, ny: int = 100, nz: int = 50, nsteps: int = 50, ninner: int = 15) -> Workload:
    """3-D 100x100x50 (5e5 cells), 400 directions, 55 band-pols, FP32 + learned guess."""
    g = Geometry(3, nx, ny, nz, 10e-9, 10e-9, 10e-9)
    uniform_walls(g, [BC_ISOTHERMAL, BC_ISOTHERMAL] + [BC_SPECULAR] * 4, [300.0, 305.0, 0, 0, 0, 0])
    return Workload(f"3d_{nx}x{ny}x{nz}_400dir_55band_fp32_learned", [g], Dirs("polar_azim", n_polar=20, n_azim=20),
                    make_bands(40, 15, 19404), 1e-12, nsteps, ninner, "fp32")


def cfg5(n_geom: int = 48, nsteps: int = 100, ninner: int = 12) -> Workload:
    """48 independent 2-D geometries, nx ~ U{32..256}, ny ~ U{32..96}, hot wall ~ U[301,320] K.

    Draws from SplitMix64(19405) in geometry order: nx, ny, T_hot.  -x wall at T_hot,
    +x wall 300 K, +-y specular, 10 nm cells.
    """
    rng = SplitMix64(19405)
    geoms = []
    for _ in range(n_geom):
        nx = rng.randint(32, 256)
        ny = rng.randint(32, 96)
        th = 301.0 + 19.0 * rng.uniform()
        g = Geometry(2, nx, ny, 1, 10e-9, 10e-9, 10e-9)
        uniform_walls(g, [BC_ISOTHERMAL, BC_ISOTHERMAL, BC_SPECULAR, BC_SPECULAR], [th, 300.0, 0, 0])
        geoms.append(g)
    return Workload(f"batch_{n_geom}x2d_400dir_55band_fp32", geoms, Dirs("polar_azim", n_polar=20, n_azim=20),
                    make_bands(40, 15, 19402), 1e-12, nsteps, ninner, "fp32")


def random_temperatures(n: int, seed: int, lo: float, hi: float) -> np.ndarray:
    """n temperatures uniform on [lo, hi) from SplitMix64(seed)."""
    rng = SplitMix64(seed)
    return np.array([lo + (hi - lo) * rng.uniform() for _ in range(n)])
