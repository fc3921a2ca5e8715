"""Python access to the plain FP64 CPU oracle (bte_oracle.c).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline / reference leg are the only callers.  The product
path (the CUDA library and its binding) never imports this module.

The shared object is compiled here with gcc (``-O2 -fopenmp
-ffp-contract=off``) the first time it is needed, or by ``build()``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "bte_oracle.c")
LIB = os.path.join(HERE, "_build", "liborc.so")

ISOTHERMAL, SPECULAR, DIFFUSE, PARTIAL, ROTATIONAL = 0, 1, 2, 3, 4
IMPLICIT, EXPLICIT, GAUSS_SEIDEL = 0, 1, 2

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/_build/liborc.so (idempotent)."""
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared", "-std=c11", SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, LIB)
    return LIB


class _Problem(C.Structure):
    _fields_ = [
        ("dim", C.c_int), ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
        ("dx", C.c_double), ("dy", C.c_double), ("dz", C.c_double),
        ("nd", C.c_int),
        ("S", C.POINTER(C.c_double)), ("w", C.POINTER(C.c_double)),
        ("rx", C.POINTER(C.c_int)), ("ry", C.POINTER(C.c_int)), ("rz", C.POINTER(C.c_int)),
        ("nb", C.c_int),
        ("wlo", C.POINTER(C.c_double)), ("whi", C.POINTER(C.c_double)), ("vg", C.POINTER(C.c_double)),
        ("beta", C.POINTER(C.c_double)), ("g", C.POINTER(C.c_double)),
        ("ngauss", C.c_int),
        ("glx", C.POINTER(C.c_double)), ("glw", C.POINTER(C.c_double)),
        ("bc_type", C.c_int * 6),
        ("bc_T", C.POINTER(C.c_double) * 6),
        ("newton_maxit", C.c_int),
        ("newton_rtol", C.c_double),
        ("beta_exp", C.c_double), ("beta_Tref", C.c_double),
        ("spec", C.c_double * 6),
    ]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(LIB)
            dp, ip = C.POINTER(C.c_double), C.POINTER(C.c_int)
            L.orc_gauss_legendre.argtypes = [C.c_int, dp, dp]
            L.orc_I0.argtypes = [C.c_int, dp, dp, dp, dp, C.c_int, dp, dp, C.c_double, dp, dp]
            L.orc_I0.restype = None
            L.orc_dirs_inplane.argtypes = [C.c_int, dp, dp, ip, ip, ip]
            L.orc_dirs_polar_azim.argtypes = [C.c_int, C.c_int, dp, dp, ip, ip, ip]
            P = C.POINTER(_Problem)
            L.orc_update_one.argtypes = [P, C.c_double, C.c_int, dp, dp, dp, dp, C.c_long, C.c_int, C.c_int, C.c_double]
            L.orc_update_one.restype = C.c_double
            L.orc_gs_update_one.argtypes = [P, C.c_double, dp, dp, dp, dp, dp, C.c_long, C.c_int, C.c_int, C.c_double]
            L.orc_gs_update_one.restype = C.c_double
            L.orc_solve_T.argtypes = [P, dp, C.c_double, C.c_double, dp]
            L.orc_cell_energy.argtypes = [P, dp, dp, dp]
            L.orc_cell_energy.restype = None
            L.orc_cell_temperatures.argtypes = [P, dp, C.c_double, C.c_double, dp, dp]
            L.orc_init_state.argtypes = [P, dp, dp, dp, dp, dp]
            L.orc_run.argtypes = [P, C.c_double, C.c_int, C.c_int, C.c_int, dp, dp, dp, dp]
            L.orc_run.restype = C.c_long
            L.orc_run_bands.argtypes = [P, C.c_int, C.c_int, C.c_double, C.c_int, C.c_int, C.c_int, dp, dp, dp, dp,
                                        SUM_FN, C.c_void_p]
            L.orc_run_bands.restype = C.c_long
            L.orc_flux.argtypes = [P, dp, dp, dp]
            L.orc_wall_I0.argtypes = [P, dp]
            L.orc_num_threads.restype = C.c_int
            U = C.POINTER(_UMesh)
            L.orc_umesh_run.argtypes = [P, U, C.c_double, C.c_int, C.c_int, C.c_int, dp, dp, dp, dp]
            L.orc_umesh_run.restype = C.c_long
            L.orc_umesh_update_one.argtypes = [P, U, C.c_double, C.c_int, dp, dp, dp, dp, C.c_long, C.c_int, C.c_int]
            L.orc_umesh_update_one.restype = C.c_double
            L.orc_umesh_wall_I0.argtypes = [P, U, dp]
            L.orc_umesh_wall_I0.restype = None
            L.orc_umesh_flux.argtypes = [P, U, dp, dp, dp]
            L.orc_umesh_flux.restype = None
            _lib = L
    return _lib


# int (*)(double* buf, long count, void* user)
SUM_FN = C.CFUNCTYPE(C.c_int, C.POINTER(C.c_double), C.c_long, C.c_void_p)


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _ip(a):
    return a.ctypes.data_as(C.POINTER(C.c_int))


def num_threads() -> int:
    return int(lib().orc_num_threads())


def gauss_legendre(n: int):
    x = np.zeros(n)
    w = np.zeros(n)
    if lib().orc_gauss_legendre(n, _dp(x), _dp(w)) != 0:
        raise ValueError("bad n")
    return x, w


def dirs_inplane(n: int):
    S = np.zeros((n, 3)); w = np.zeros(n)
    r = np.zeros((3, n), dtype=np.int32)
    if lib().orc_dirs_inplane(n, _dp(S), _dp(w), _ip(r[0]), _ip(r[1]), _ip(r[2])) != 0:
        raise ValueError("in-plane set needs n % 4 == 0")
    return S, w, r


def dirs_polar_azim(ntheta: int, nphi: int):
    n = ntheta * nphi
    S = np.zeros((n, 3)); w = np.zeros(n)
    r = np.zeros((3, n), dtype=np.int32)
    if lib().orc_dirs_polar_azim(ntheta, nphi, _dp(S), _dp(w), _ip(r[0]), _ip(r[1]), _ip(r[2])) != 0:
        raise ValueError("polar x azimuthal set needs even ntheta and nphi % 4 == 0")
    return S, w, r


def dirs_for(spec):
    """Direction tables for a direction-set description (attributes kind, n_inplane, n_polar, n_azim)."""
    if spec.kind == "inplane":
        return dirs_inplane(spec.n_inplane)
    return dirs_polar_azim(spec.n_polar, spec.n_azim)


def I0(bands, T: float, ngauss: int = 16):
    """(I0_b(T), dI0_b/dT) for every band."""
    x, w = gauss_legendre(ngauss)
    nb = len(bands.vg)
    out = np.zeros(nb); d = np.zeros(nb)
    arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (bands.omega_lo, bands.omega_hi, bands.vg, bands.degeneracy)]
    lib().orc_I0(nb, _dp(arrs[0]), _dp(arrs[1]), _dp(arrs[2]), _dp(arrs[3]), ngauss, _dp(x), _dp(w), float(T), _dp(out), _dp(d))
    return out, d


class Problem:
    """One structured geometry with its direction set, bands and walls.

    ``geom`` needs dim, nx, ny, nz, dx, dy, dz and bc (a list of (kind, per-face
    temperatures or None) per side); ``bands`` needs omega_lo, omega_hi, vg,
    beta, degeneracy.  ``dirs`` is (S[nd,3], w[nd], r[3,nd]) -- any table,
    so tests may permute or hand-build direction sets.
    """

    def __init__(self, geom, dirs, bands, ngauss: int = 16, newton_rtol: float = 1e-14, newton_maxit: int = 50,
                 beta_exp: float = 0.0, beta_Tref: float = 300.0):
        """beta_exp != 0: beta_b(T) = beta_b (T_p / beta_Tref)^beta_exp per cell."""
        self.geom = geom
        S, w, r = dirs
        self.S = np.ascontiguousarray(S, dtype=np.float64)
        self.w = np.ascontiguousarray(w, dtype=np.float64)
        self.r = np.ascontiguousarray(r, dtype=np.int32)
        self.nd = int(self.w.shape[0])
        self.bands = [np.ascontiguousarray(a, dtype=np.float64) for a in
                      (bands.omega_lo, bands.omega_hi, bands.vg, bands.beta, bands.degeneracy)]
        self.nb = int(self.bands[2].shape[0])
        self.glx, self.glw = gauss_legendre(ngauss)
        self.bcT = []
        p = _Problem()
        p.dim, p.nx, p.ny, p.nz = geom.dim, geom.nx, geom.ny, geom.nz
        p.dx, p.dy, p.dz = geom.dx, geom.dy, geom.dz
        p.nd = self.nd
        p.S, p.w = _dp(self.S), _dp(self.w)
        p.rx, p.ry, p.rz = _ip(self.r[0]), _ip(self.r[1]), _ip(self.r[2])
        p.nb = self.nb
        p.wlo, p.whi, p.vg, p.beta, p.g = (_dp(a) for a in self.bands)
        p.ngauss = ngauss
        p.glx, p.glw = _dp(self.glx), _dp(self.glw)
        for s in range(6):
            if s < 2 * geom.dim and geom.bc[s][0] == ISOTHERMAL:
                T = np.ascontiguousarray(geom.bc[s][1], dtype=np.float64)
                self.bcT.append(T)
                p.bc_type[s] = ISOTHERMAL
                p.bc_T[s] = _dp(T)
            else:
                kind = geom.bc[s][0] if s < 2 * geom.dim else SPECULAR
                p.bc_type[s] = kind if kind in (DIFFUSE, PARTIAL) else SPECULAR
                p.bc_T[s] = C.POINTER(C.c_double)()
                if kind == PARTIAL:  # (PARTIAL, specularity)
                    p.spec[s] = float(geom.bc[s][1])
        p.newton_maxit = newton_maxit
        p.newton_rtol = newton_rtol
        p.beta_exp = float(beta_exp)
        p.beta_Tref = float(beta_Tref)
        self._p = p
        self.nc = geom.nx * geom.ny * geom.nz

    @property
    def ptr(self):
        return C.byref(self._p)

    # -- state ---------------------------------------------------------------
    def init_state(self, T_cells):
        T = np.ascontiguousarray(np.broadcast_to(np.asarray(T_cells, dtype=np.float64), (self.nc,)))
        st = {
            "I": np.zeros((self.nc, self.nd, self.nb)),
            "Tp": np.zeros(self.nc), "TL": np.zeros(self.nc), "I0": np.zeros((self.nc, self.nb)),
        }
        lib().orc_init_state(self.ptr, _dp(T), _dp(st["I"]), _dp(st["Tp"]), _dp(st["TL"]), _dp(st["I0"]))
        return st

    def run(self, st, dt: float, nsteps: int, ninner: int, scheme: int = IMPLICIT) -> int:
        r = lib().orc_run(self.ptr, float(dt), int(nsteps), int(ninner), int(scheme),
                          _dp(st["I"]), _dp(st["Tp"]), _dp(st["TL"]), _dp(st["I0"]))
        if r < 0:
            raise RuntimeError("oracle: a cell has no temperature in [1, 5000] K")
        return int(r)

    def run_bands(self, st, b0: int, b1: int, total, dt: float, nsteps: int, ninner: int,
                  scheme: int = IMPLICIT) -> int:
        """The time loop over bands [b0, b1) only (Sec. 3.3 band partition).
        total(E) receives the (ncells, 2) partial energies [E_L, E_p] of these
        bands and returns their totals over all band owners (same shape)."""
        def cb(buf, count, user):
            try:
                E = np.ctypeslib.as_array(buf, shape=(count,)).reshape(-1, 2)
                E[:] = total(E.copy())
                return 0
            except Exception:
                import traceback
                traceback.print_exc()
                return 1
        fn = SUM_FN(cb)
        r = lib().orc_run_bands(self.ptr, int(b0), int(b1), float(dt), int(nsteps), int(ninner), int(scheme),
                                _dp(st["I"]), _dp(st["Tp"]), _dp(st["TL"]), _dp(st["I0"]), fn, None)
        if r == -2:
            raise RuntimeError("oracle: the band-sum callback failed")
        if r < 0:
            raise RuntimeError("oracle: a cell has no temperature in [1, 5000] K (or a bad band range)")
        return int(r)

    # -- pieces used by sampled checks ---------------------------------------
    def wall_I0(self):
        nf = sum(self.geom.nfaces(s) for s in range(2 * self.geom.dim))
        out = np.zeros((max(nf, 1), self.nb))
        lib().orc_wall_I0(self.ptr, _dp(out))
        return out

    def update_one(self, dt, scheme, In, Ik, I0cells, I0wall, P, d, b, bscale=1.0) -> float:
        """bscale: beta_b(T_p)/beta_b of cell P (1 when tau does not depend on T)."""
        return float(lib().orc_update_one(self.ptr, float(dt), int(scheme), _dp(In), _dp(Ik), _dp(I0cells),
                                          _dp(I0wall), int(P), int(d), int(b), float(bscale)))

    def gs_update_one(self, dt, In, Ik, Inew, I0cells, I0wall, P, d, b, bscale=1.0) -> float:
        """Sweep-ordered update of (P, d, b): interior upwind values from Inew."""
        return float(lib().orc_gs_update_one(self.ptr, float(dt), _dp(In), _dp(Ik), _dp(Inew), _dp(I0cells),
                                             _dp(I0wall), int(P), int(d), int(b), float(bscale)))

    def cell_energy(self, row):
        row = np.ascontiguousarray(row, dtype=np.float64)
        EL = C.c_double(); Ep = C.c_double()
        lib().orc_cell_energy(self.ptr, _dp(row), C.byref(EL), C.byref(Ep))
        return EL.value, Ep.value

    def cell_temperatures(self, row, Tp_guess=300.0, TL_guess=300.0):
        row = np.ascontiguousarray(row, dtype=np.float64)
        Tp = C.c_double(); TL = C.c_double()
        s = lib().orc_cell_temperatures(self.ptr, _dp(row), float(Tp_guess), float(TL_guess), C.byref(Tp), C.byref(TL))
        if s < 0:
            raise RuntimeError("oracle: no temperature in [1, 5000] K")
        return Tp.value, TL.value

    def solve_T(self, a, E, T_guess=300.0):
        a = np.ascontiguousarray(a, dtype=np.float64)
        T = C.c_double()
        s = lib().orc_solve_T(self.ptr, _dp(a), float(E), float(T_guess), C.byref(T))
        return T.value, int(s)

    def flux(self, I):
        I = np.ascontiguousarray(I, dtype=np.float64)
        q = np.zeros((self.nc, self.geom.dim))
        qw = np.zeros(6)
        lib().orc_flux(self.ptr, _dp(I), _dp(q), _dp(qw))
        return q, qw[: 2 * self.geom.dim]


class _UMesh(C.Structure):
    _fields_ = [("dim", C.c_int), ("nc", C.c_long), ("nf", C.c_long), ("vol", C.POINTER(C.c_double)),
                ("owner", C.POINTER(C.c_long)), ("nbr", C.POINTER(C.c_long)), ("nA", C.POINTER(C.c_double)),
                ("btype", C.POINTER(C.c_int)), ("Twall", C.POINTER(C.c_double)), ("spec", C.POINTER(C.c_double)),
                ("rot_angle", C.c_double), ("fc", C.POINTER(C.c_double)), ("rot_map", C.POINTER(C.c_int))]


class UMeshProblem:
    """An unstructured mesh (paper_2305_19400_gb300.mesh.UMesh face list) with
    its direction set, bands and boundary conditions.

    bc: {tag: (kind, T)} with kind ISOTHERMAL (T a float, or an array over the
    mesh's faces indexed by face id), SPECULAR or DIFFUSE (T ignored),
    PARTIAL (T the specularity p in [0, 1], a float or an array over the
    faces), or ROTATIONAL (T the wedge angle of an axisymmetric problem about
    the z axis; every ROTATIONAL tag takes the same angle).  The direction and
    band tables live in a Problem on a one-cell grid."""

    def __init__(self, mesh, dirs, bands, bc, ngauss: int = 16, newton_rtol: float = 1e-14, newton_maxit: int = 50,
                 beta_exp: float = 0.0, beta_Tref: float = 300.0):
        class _G:  # one-cell placeholder grid for the tables
            pass
        g = _G()
        g.dim, g.nx, g.ny, g.nz, g.dx, g.dy, g.dz = mesh.dim, 1, 1, 1, 1.0, 1.0, 1.0
        g.bc = [(SPECULAR, None)] * (2 * mesh.dim)
        self.tables = Problem(g, dirs, bands, ngauss, newton_rtol, newton_maxit, beta_exp, beta_Tref)
        self.mesh = mesh
        self.nd, self.nb, self.nc = self.tables.nd, self.tables.nb, mesh.ncells
        nf = mesh.nfaces
        self.vol = np.ascontiguousarray(mesh.volume, dtype=np.float64)
        self.owner = np.ascontiguousarray(mesh.owner, dtype=np.int64)
        self.nbr = np.ascontiguousarray(mesh.neighbor, dtype=np.int64)
        self.nA = np.ascontiguousarray(mesh.nA, dtype=np.float64)
        self.btype = np.full(nf, SPECULAR, dtype=np.int32)
        self.Twall = np.zeros(nf)
        self.spec = np.zeros(nf)
        self.fc = np.ascontiguousarray(mesh.face_center, dtype=np.float64)
        rot_angle = 0.0
        for f in np.nonzero(self.nbr < 0)[0]:
            kind, T = bc[int(mesh.tag[f])]
            self.btype[f] = kind
            if kind == ISOTHERMAL:
                self.Twall[f] = T if np.isscalar(T) else T[f]
            elif kind == PARTIAL:
                self.spec[f] = T if np.isscalar(T) else T[f]
            elif kind == ROTATIONAL:
                rot_angle = float(T)
        m = _UMesh()
        m.dim, m.nc, m.nf = mesh.dim, self.nc, nf
        m.vol, m.nA, m.Twall, m.spec = _dp(self.vol), _dp(self.nA), _dp(self.Twall), _dp(self.spec)
        m.rot_angle, m.fc = rot_angle, _dp(self.fc)
        m.owner = self.owner.ctypes.data_as(C.POINTER(C.c_long))
        m.nbr = self.nbr.ctypes.data_as(C.POINTER(C.c_long))
        m.btype = _ip(self.btype)
        self._m = m

    @property
    def ptr(self):
        return C.byref(self._m)

    def init_state(self, T_cells):
        T = np.ascontiguousarray(np.broadcast_to(np.asarray(T_cells, dtype=np.float64), (self.nc,)))
        st = {"I": np.zeros((self.nc, self.nd, self.nb)), "Tp": T.copy(), "TL": T.copy(),
              "I0": np.zeros((self.nc, self.nb))}
        for P in range(self.nc):
            st["I0"][P] = I0(_BandView(self.tables), T[P], len(self.tables.glx))[0]
            st["I"][P] = st["I0"][P][None, :]
        return st

    def run(self, st, dt, nsteps, ninner, scheme=IMPLICIT) -> int:
        r = lib().orc_umesh_run(self.tables.ptr, self.ptr, float(dt), int(nsteps), int(ninner), int(scheme),
                                _dp(st["I"]), _dp(st["Tp"]), _dp(st["TL"]), _dp(st["I0"]))
        if r == -2:
            raise RuntimeError("oracle: the wedge angle is not a rotation symmetry of the direction set")
        if r < 0:
            raise RuntimeError("oracle: a cell has no temperature in [1, 5000] K")
        return int(r)

    def wall_I0(self):
        out = np.zeros((max(self.mesh.nfaces, 1), self.nb))
        lib().orc_umesh_wall_I0(self.tables.ptr, self.ptr, _dp(out))
        return out

    def update_one(self, dt, scheme, In, Ik, I0cells, I0wall, P, d, b) -> float:
        return float(lib().orc_umesh_update_one(self.tables.ptr, self.ptr, float(dt), int(scheme), _dp(In), _dp(Ik),
                                                _dp(I0cells), _dp(I0wall), int(P), int(d), int(b)))

    def flux(self, I):
        """(q[nc, 3] per cell, Q[nfaces] net outflow per boundary face)."""
        I = np.ascontiguousarray(I, dtype=np.float64)
        q = np.zeros((self.nc, 3)); Q = np.zeros(self.mesh.nfaces)
        lib().orc_umesh_flux(self.tables.ptr, self.ptr, _dp(I), _dp(q), _dp(Q))
        return q, Q

    def cell_energy(self, row):
        return self.tables.cell_energy(row)


class _BandView:
    """The band arrays of a Problem in the attribute form I0() takes."""

    def __init__(self, prob):
        self.omega_lo, self.omega_hi, self.vg, self.beta, self.degeneracy = prob.bands
