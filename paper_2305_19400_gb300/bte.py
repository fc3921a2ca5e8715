"""Thin Python binding of libbte (include/bte.h): same entry-point names,
argument marshalling only.  Every step of the hot path runs in the library's
CUDA kernels; there is no CPU fallback.  PyTorch supplies device memory
(workspace, device-side outputs) and the CUDA stream.

Loading fails loudly (RuntimeError) when libbte.so has not been built.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libbte.so")

BTE_OK, BTE_W_FALLBACK = 0, 1
BTE_E = {-1: "BTE_E_ARG", -2: "BTE_E_STATE", -3: "BTE_E_CUDA", -4: "BTE_E_NOMEM", -5: "BTE_E_NONFINITE",
         -6: "BTE_E_TIMEOUT", -7: "BTE_E_EXCHANGE"}
(BTE_E_ARG, BTE_E_STATE, BTE_E_CUDA, BTE_E_NOMEM, BTE_E_NONFINITE, BTE_E_TIMEOUT,
 BTE_E_EXCHANGE) = -1, -2, -3, -4, -5, -6, -7
BTE_DIRS_INPLANE, BTE_DIRS_POLAR_AZIM = 0, 1
BTE_FP64, BTE_FP32, BTE_BF16 = 0, 1, 2
BTE_BC_ISOTHERMAL, BTE_BC_SPECULAR, BTE_BC_DIFFUSE, BTE_BC_PARTIAL, BTE_BC_ROTATIONAL = 0, 1, 2, 3, 4
BTE_IMPLICIT_JACOBI, BTE_EXPLICIT, BTE_IMPLICIT_GS = 0, 1, 2
BTE_T_PSEUDO, BTE_T_LATTICE, BTE_E_LATTICE = 0, 1, 2


class bte_geom(C.Structure):
    _fields_ = [("dim", C.c_int), ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("dx", C.c_double), ("dy", C.c_double), ("dz", C.c_double)]


class bte_opts(C.Structure):
    _fields_ = [("dir_kind", C.c_int), ("n_inplane", C.c_int), ("n_polar", C.c_int), ("n_azim", C.c_int),
                ("precision", C.c_int), ("learned", C.c_int), ("n_gauss", C.c_int), ("newton_rtol", C.c_double),
                ("newton_maxit", C.c_int), ("cuda_stream", C.c_void_p), ("T_ref", C.c_double),
                ("use_graph", C.c_int), ("autotune", C.c_int), ("beta_T_exp", C.c_double),
                ("fp64_strict", C.c_int)]


class bte_stats(C.Structure):
    _fields_ = [("updates", C.c_longlong), ("solve_evals", C.c_longlong), ("solves", C.c_longlong),
                ("fallbacks", C.c_longlong), ("nonfinite", C.c_longlong), ("launches", C.c_int),
                ("gpu_ms", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class bte_umesh_desc(C.Structure):
    _fields_ = [("dim", C.c_int), ("ncells", C.c_longlong), ("nfaces", C.c_longlong),
                ("volume", C.POINTER(C.c_double)), ("owner", C.POINTER(C.c_longlong)),
                ("neighbor", C.POINTER(C.c_longlong)), ("nA", C.POINTER(C.c_double)), ("tag", C.POINTER(C.c_int)),
                ("fc", C.POINTER(C.c_double))]


# Every symbol include/bte.h and include/bte_umesh.h declare, with its ctypes signature.
_dp, _ip, _vp, _h = C.POINTER(C.c_double), C.POINTER(C.c_int), C.c_void_p, C.c_void_p
# int (*)(double* buf, long long count, void* cuda_stream, void* user)
bte_allreduce_fn = C.CFUNCTYPE(C.c_int, C.c_void_p, C.c_longlong, C.c_void_p, C.c_void_p)
SIGNATURES = {
    "bte_default_opts": (C.c_int, [C.POINTER(bte_opts)]),
    "bte_init_mesh": (C.c_int, [C.POINTER(_h), C.c_int, C.POINTER(bte_geom), C.POINTER(bte_opts)]),
    "bte_set_bands": (C.c_int, [_h, C.c_int, _dp, _dp, _dp, _dp, _dp]),
    "bte_set_band_range": (C.c_int, [_h, C.c_int, C.c_int]),
    "bte_set_exchange": (C.c_int, [_h, bte_allreduce_fn, _vp, _vp]),
    "bte_workspace_bytes": (C.c_size_t, [_h]),
    "bte_bind_workspace": (C.c_int, [_h, _vp, C.c_size_t]),
    "bte_set_bc": (C.c_int, [_h, C.c_int, C.c_int, C.c_int, _dp, C.c_double]),
    "bte_set_specularity": (C.c_int, [_h, C.c_int, C.c_int, C.c_double]),
    "bte_set_initial": (C.c_int, [_h, C.c_int, _dp, C.c_double]),
    "bte_step": (C.c_int, [_h, C.c_double, C.c_int, C.c_int, C.c_int, C.POINTER(bte_stats)]),
    "bte_autotune": (C.c_int, [_h, C.c_double, C.c_int, C.c_char_p, C.c_size_t]),
    "bte_get_T": (C.c_int, [_h, C.c_int, C.c_int, _vp, C.c_int]),
    "bte_get_flux": (C.c_int, [_h, C.c_int, _vp, _vp, C.c_int]),
    "bte_get_intensity": (C.c_int, [_h, C.c_int, _vp, C.c_int]),
    "bte_set_intensity": (C.c_int, [_h, C.c_int, _vp, _vp, C.c_int]),
    "bte_get_directions": (C.c_int, [_h, _dp, _dp, _ip]),
    "bte_get_wall_flux_noalloc": (C.c_int, [_h, C.c_int, _vp, C.c_int]),
    "bte_measure_peak": (C.c_int, [C.c_int, _dp, _dp]),
    "bte_set_sweep_timing": (C.c_int, [_h, C.c_int]),
    "bte_sweep_times": (C.c_int, [_h, C.POINTER(C.c_float), C.c_int]),
    "bte_train_mlp": (C.c_int, [_h, C.c_longlong, C.c_double, C.c_double, C.c_int, C.c_ulonglong, _dp]),
    "bte_mlp_params": (C.c_int, [_h, C.c_int, C.POINTER(C.c_float), C.c_int]),
    "bte_mlp_set_params": (C.c_int, [_h, C.c_int, C.POINTER(C.c_float), C.c_int]),
    "bte_mlp_grad": (C.c_int, [_h, C.c_int, C.POINTER(C.c_float), C.POINTER(C.c_float), C.c_int,
                               C.POINTER(C.c_float), _dp]),
    "bte_solve_T": (C.c_int, [_h, _dp, _dp, C.c_int, C.c_int, _dp, _ip]),
    "bte_destroy": (C.c_int, [_h]),
    "bte_last_error": (C.c_char_p, [_h]),
    "bte_umesh_create": (C.c_int, [C.POINTER(bte_umesh_desc), C.POINTER(bte_opts), C.POINTER(_h)]),
    "bte_umesh_set_bands": (C.c_int, [_h, C.c_int, _dp, _dp, _dp, _dp, _dp]),
    "bte_umesh_set_bc": (C.c_int, [_h, C.c_int, C.c_int, _dp, C.c_double]),
    "bte_umesh_set_initial": (C.c_int, [_h, _dp, C.c_double]),
    "bte_umesh_step": (C.c_int, [_h, C.c_double, C.c_int, C.c_int, C.c_int, C.POINTER(bte_stats)]),
    "bte_umesh_get_T": (C.c_int, [_h, C.c_int, _vp, C.c_int]),
    "bte_umesh_get_intensity": (C.c_int, [_h, _dp]),
    "bte_umesh_get_flux": (C.c_int, [_h, _dp, _dp]),
    "bte_umesh_set_intensity": (C.c_int, [_h, _dp, _dp]),
    "bte_umesh_last_error": (C.c_char_p, [_h]),
    "bte_umesh_destroy": (None, [_h]),
}

_lib = None


def lib():
    """The loaded libbte.so (RuntimeError if it is missing)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libbte.so is not built ({LIB_PATH}); run paper_2305_19400_gb300.build.build()")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


class BTEError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{BTE_E.get(code, code)}: {msg}")
        self.code = code


def _check(h, rc):
    if rc < 0:
        msg = lib().bte_last_error(h)
        raise BTEError(rc, msg.decode() if msg else "")
    return rc


def _ptr(x):
    """Host numpy array -> double*, torch tensor -> device/host address, None -> NULL."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        return C.c_void_p(x.ctypes.data)
    return C.c_void_p(x.data_ptr())


# ---- entry points with the C names -----------------------------------------
def bte_default_opts():
    o = bte_opts()
    lib().bte_default_opts(C.byref(o))
    return o


def bte_init_mesh(geoms, opts=None):
    arr = (bte_geom * len(geoms))(*geoms)
    h = C.c_void_p()
    rc = lib().bte_init_mesh(C.byref(h), len(geoms), arr, C.byref(opts) if opts is not None else None)
    _check(None, rc)
    return h


def bte_set_bands(h, omega_lo, omega_hi, vg, beta, degeneracy):
    arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (omega_lo, omega_hi, vg, beta, degeneracy)]
    return _check(h, lib().bte_set_bands(h, len(arrs[0]), *[a.ctypes.data_as(_dp) for a in arrs]))


def bte_set_band_range(h, band_lo, band_hi):
    return _check(h, lib().bte_set_band_range(h, int(band_lo), int(band_hi)))


def bte_set_exchange(h, fn, dev_buf=None):
    """fn(buf_ptr, count, stream_ptr) -> int, called from bte_step.  Returns the
    ctypes callback object, which the caller must keep alive while stepping."""
    def tramp(buf, count, stream, user):
        try:
            return int(fn(buf, count, stream) or 0)
        except Exception:  # an exception cannot cross the C frame: report it as a failed exchange
            import traceback
            traceback.print_exc()
            return 1
    cb = bte_allreduce_fn(tramp)
    _check(h, lib().bte_set_exchange(h, cb, None, _ptr(dev_buf)))
    return cb


def bte_workspace_bytes(h):
    return int(lib().bte_workspace_bytes(h))


def bte_bind_workspace(h, tensor):
    return _check(h, lib().bte_bind_workspace(h, C.c_void_p(tensor.data_ptr()), tensor.numel() * tensor.element_size()))


def bte_set_bc(h, geom, side, kind, T_faces=None, T_uniform=300.0):
    arr = None if T_faces is None else np.ascontiguousarray(T_faces, dtype=np.float64)
    return _check(h, lib().bte_set_bc(h, geom, side, kind, None if arr is None else arr.ctypes.data_as(_dp), float(T_uniform)))


def bte_set_initial(h, geom, T_cells=None, T_uniform=300.0):
    arr = None if T_cells is None else np.ascontiguousarray(T_cells, dtype=np.float64)
    return _check(h, lib().bte_set_initial(h, geom, None if arr is None else arr.ctypes.data_as(_dp), float(T_uniform)))


def bte_step(h, dt, nsteps, ninner, scheme=BTE_IMPLICIT_JACOBI, want_stats=True):
    st = bte_stats() if want_stats else None
    rc = lib().bte_step(h, float(dt), int(nsteps), int(ninner), int(scheme), C.byref(st) if st is not None else None)
    _check(h, rc)
    return rc, (st.as_dict() if st is not None else None)


def bte_autotune(h, dt, scheme=BTE_IMPLICIT_JACOBI):
    buf = C.create_string_buffer(4096)
    _check(h, lib().bte_autotune(h, float(dt), int(scheme), buf, 4096))
    return buf.value.decode()


def bte_get_T(h, geom, which, out):
    """out: float64 numpy array (host) or torch CUDA tensor (device)."""
    on_dev = 0 if isinstance(out, np.ndarray) else 1
    return _check(h, lib().bte_get_T(h, geom, which, _ptr(out), on_dev))


def bte_get_flux(h, geom, q_cells=None, q_walls=None, on_device=False):
    return _check(h, lib().bte_get_flux(h, geom, _ptr(q_cells), _ptr(q_walls), 1 if on_device else 0))


def bte_get_intensity(h, geom, out):
    on_dev = 0 if isinstance(out, np.ndarray) else 1
    return _check(h, lib().bte_get_intensity(h, geom, _ptr(out), on_dev))


def bte_set_intensity(h, geom, I, Tp):
    on_dev = 0 if isinstance(I, np.ndarray) else 1
    if on_dev == 0:
        I = np.ascontiguousarray(I, dtype=np.float64)
        Tp = np.ascontiguousarray(Tp, dtype=np.float64)
    return _check(h, lib().bte_set_intensity(h, geom, _ptr(I), _ptr(Tp), on_dev))


def bte_get_directions(h):
    nd = _check(h, lib().bte_get_directions(h, None, None, None))
    S = np.zeros((nd, 3)); w = np.zeros(nd); r = np.zeros((3, nd), dtype=np.int32)
    lib().bte_get_directions(h, S.ctypes.data_as(_dp), w.ctypes.data_as(_dp), r.ctypes.data_as(_ip))
    return S, w, r


def bte_get_wall_flux_noalloc(h, geom, q_walls):
    """q_walls: float64 numpy array (host) or torch CUDA tensor (device), 2*dim values."""
    on_dev = 0 if isinstance(q_walls, np.ndarray) else 1
    return _check(h, lib().bte_get_wall_flux_noalloc(h, geom, _ptr(q_walls), on_dev))


def bte_train_mlp(h, n_pairs, T_lo, T_hi, epochs, seed=1):
    loss = np.zeros(2)
    _check(h, lib().bte_train_mlp(h, int(n_pairs), float(T_lo), float(T_hi), int(epochs), int(seed),
                                  loss.ctypes.data_as(_dp)))
    return loss


def _fp(a):
    return a.ctypes.data_as(C.POINTER(C.c_float))


def bte_mlp_params(h, net):
    n = _check(h, lib().bte_mlp_params(h, int(net), None, 0))
    out = np.zeros(n, dtype=np.float32)
    _check(h, lib().bte_mlp_params(h, int(net), _fp(out), n))
    return out


def bte_mlp_set_params(h, net, params):
    p = np.ascontiguousarray(params, dtype=np.float32)
    return _check(h, lib().bte_mlp_set_params(h, int(net), _fp(p), p.size))


def bte_mlp_grad(h, net, x, y):
    """x: (n,), y: (k, n) float32; returns (grad, loss)."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    y = np.ascontiguousarray(y, dtype=np.float32)
    n = x.size
    g = np.zeros(_check(h, lib().bte_mlp_params(h, int(net), None, 0)), dtype=np.float32)
    loss = C.c_double()
    _check(h, lib().bte_mlp_grad(h, int(net), _fp(x), _fp(y), n, _fp(g), C.byref(loss)))
    return g, loss.value


def bte_solve_T(h, Ep, T0=None, learned=False):
    Ep = np.ascontiguousarray(Ep, dtype=np.float64)
    n = Ep.size
    T = np.zeros(n)
    ev = np.zeros(n, dtype=np.int32)
    t0 = None if T0 is None else np.ascontiguousarray(T0, dtype=np.float64)
    _check(h, lib().bte_solve_T(h, Ep.ctypes.data_as(_dp), None if t0 is None else t0.ctypes.data_as(_dp), n,
                                1 if learned else 0, T.ctypes.data_as(_dp), ev.ctypes.data_as(_ip)))
    return T, ev


def bte_set_sweep_timing(h, on=True):
    return _check(h, lib().bte_set_sweep_timing(h, 1 if on else 0))


def bte_sweep_times(h):
    """Device time (ms) of each sweep launch of the most recent time step."""
    n = _check(h, lib().bte_sweep_times(h, None, 0))
    ms = np.zeros(n, dtype=np.float32)
    _check(h, lib().bte_sweep_times(h, ms.ctypes.data_as(C.POINTER(C.c_float)), n))
    return ms.astype(np.float64)


BTE_PEAK_FP64_FMA, BTE_PEAK_FP32X2_FMA = 0, 1


def bte_measure_peak(kind):
    """(flop/s, ms of the timed launch) of the FMA loop of `kind` on the current device."""
    f = np.zeros(1)
    ms = np.zeros(1)
    rc = lib().bte_measure_peak(int(kind), f.ctypes.data_as(_dp), ms.ctypes.data_as(_dp))
    if rc < 0:
        raise BTEError(rc, "bte_measure_peak failed")
    return float(f[0]), float(ms[0])


def bte_destroy(h):
    return _check(None, lib().bte_destroy(h))


def bte_last_error(h):
    m = lib().bte_last_error(h)
    return m.decode() if m else ""


def allreduce_exchange(group=None):
    """Exchange for band-range handles (Sec. 3.3): sums a float64 tensor of
    per-cell (E_L, E_p) partials in place over the ranks of a torch.distributed
    group.  NCCL reduces the device tensor on the current stream; other
    backends (gloo) reduce a host copy."""
    import torch
    import torch.distributed as dist

    def fn(buf):
        if buf.is_cuda and dist.get_backend(group) != "nccl":
            host = buf.cpu()
            dist.all_reduce(host, group=group)
            buf.copy_(host)
        else:
            dist.all_reduce(buf, group=group)
    return fn


# ---- convenience: a solver built from a workload description ---------------
class Solver:
    """Marshals a workload (paper_2305_19400_gb300.workloads) into the C calls.

    Device memory comes from a torch uint8 tensor bound as the workspace; the
    stream is the given torch stream (default: torch's current stream).
    """

    def __init__(self, workload, precision=BTE_FP64, stream=None, bind_workspace=True, n_gauss=16, T_init=None,
                 use_graph=False, autotune=False, learned=False, band_range=None, exchange=None, beta_exp=0.0,
                 T_ref=None, fp64_strict=False):
        """band_range=(lo, hi) stores and sweeps only bands [lo, hi); exchange(buf)
        then sums the float64 CUDA tensor buf of per-cell (E_L, E_p) partials
        over the ranks in place (e.g. allreduce_exchange()); it runs with this
        solver's stream current."""
        import torch

        self.wl = workload
        self.torch = torch
        o = bte_default_opts()
        d = workload.dirs
        if d.kind == "inplane":
            o.dir_kind, o.n_inplane = BTE_DIRS_INPLANE, d.n_inplane
        else:
            o.dir_kind, o.n_polar, o.n_azim = BTE_DIRS_POLAR_AZIM, d.n_polar, d.n_azim
        o.precision = precision
        o.n_gauss = n_gauss
        o.use_graph = 1 if use_graph else 0
        o.learned = 1 if learned else 0
        o.autotune = 1 if autotune else 0
        o.beta_T_exp = float(beta_exp)
        o.fp64_strict = 1 if fp64_strict else 0
        if T_ref is not None:
            o.T_ref = float(T_ref)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        o.cuda_stream = self.stream.cuda_stream
        geoms = [bte_geom(g.dim, g.nx, g.ny, g.nz, g.dx, g.dy, g.dz) for g in workload.geoms]
        self.h = bte_init_mesh(geoms, o)
        b = workload.bands
        bte_set_bands(self.h, b.omega_lo, b.omega_hi, b.vg, b.beta, b.degeneracy)
        self.band_range = (0, b.nb) if band_range is None else tuple(int(x) for x in band_range)
        if band_range is not None:
            bte_set_band_range(self.h, *self.band_range)
        if exchange is not None:
            ncells = sum(g.ncells for g in workload.geoms)
            self.xbuf = torch.empty(2 * ncells, dtype=torch.float64, device="cuda")

            def run_exchange(buf_ptr, count, stream_ptr):
                with torch.cuda.stream(self.stream):
                    exchange(self.xbuf)
                return 0
            self._xcb = bte_set_exchange(self.h, run_exchange, self.xbuf)
        self.ws = None
        if bind_workspace:
            nbytes = bte_workspace_bytes(self.h)
            self.ws = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
            off = (-self.ws.data_ptr()) % 256
            self.ws_view = self.ws[off:off + nbytes]
            bte_bind_workspace(self.h, self.ws_view)
        for gi, g in enumerate(workload.geoms):
            for side, (kind, T) in enumerate(g.bc):
                if kind == BTE_BC_PARTIAL:  # (BTE_BC_PARTIAL, specularity)
                    _check(self.h, lib().bte_set_specularity(self.h, gi, side, float(T)))
                else:
                    bte_set_bc(self.h, gi, side, kind, T, 300.0)
            bte_set_initial(self.h, gi, None if T_init is None else T_init[gi], g.T_init)

    def step(self, nsteps=None, ninner=None, dt=None, scheme=BTE_IMPLICIT_JACOBI, want_stats=True):
        wl = self.wl
        return bte_step(self.h, wl.dt if dt is None else dt, wl.nsteps if nsteps is None else nsteps,
                        wl.ninner if ninner is None else ninner, scheme, want_stats)

    def T(self, geom=0, which=BTE_T_LATTICE):
        g = self.wl.geoms[geom]
        out = np.zeros(g.ncells)
        bte_get_T(self.h, geom, which, out)
        return out

    def intensity(self, geom=0):
        g = self.wl.geoms[geom]
        out = np.zeros((g.ncells, self.wl.dirs.nd, self.band_range[1] - self.band_range[0]))
        bte_get_intensity(self.h, geom, out)
        return out

    def flux(self, geom=0):
        g = self.wl.geoms[geom]
        q = np.zeros((g.ncells, g.dim))
        qw = np.zeros(2 * g.dim)
        bte_get_flux(self.h, geom, q, qw)
        return q, qw

    def close(self):
        if self.h is not None:
            bte_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------- unstructured meshes
def _ucheck(u, rc):
    if rc < 0:
        msg = lib().bte_umesh_last_error(u)
        raise BTEError(rc, msg.decode() if msg else "")
    return rc


class UMeshSolver:
    """Marshals an unstructured mesh (paper_2305_19400_gb300.mesh.UMesh face
    list), a direction set and a band table into the bte_umesh_* calls.

    bc: {tag: (kind, T)} with kind BTE_BC_ISOTHERMAL (T a float, or an array
    over the mesh's faces indexed by face id), BTE_BC_SPECULAR or
    BTE_BC_DIFFUSE (T ignored), BTE_BC_PARTIAL (T the specularity p, a
    float or an array over the faces), or BTE_BC_ROTATIONAL (T the wedge
    angle of an axisymmetric mesh, mesh.wedge_ring).  beta_exp: relaxation
    rates beta_b (T_p / T_ref)^beta_exp per cell (0: tau fixed)."""

    def __init__(self, mesh, dirs, bands, bc, T_init=None, stream=None, n_gauss=16, precision=BTE_FP64,
                 beta_exp=0.0, T_ref=300.0):
        import torch
        o = bte_default_opts()
        o.precision = precision
        o.beta_T_exp = beta_exp
        o.T_ref = T_ref
        if dirs.kind == "inplane":
            o.dir_kind, o.n_inplane = BTE_DIRS_INPLANE, dirs.n_inplane
        else:
            o.dir_kind, o.n_polar, o.n_azim = BTE_DIRS_POLAR_AZIM, dirs.n_polar, dirs.n_azim
        o.n_gauss = n_gauss
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        o.cuda_stream = self.stream.cuda_stream
        self.mesh, self.dirs, self.bands = mesh, dirs, bands
        self._keep = [np.ascontiguousarray(mesh.volume, dtype=np.float64),
                      np.ascontiguousarray(mesh.owner, dtype=np.int64),
                      np.ascontiguousarray(mesh.neighbor, dtype=np.int64),
                      np.ascontiguousarray(mesh.nA, dtype=np.float64),
                      np.ascontiguousarray(mesh.tag, dtype=np.int32),
                      np.ascontiguousarray(mesh.face_center, dtype=np.float64)]
        vol, own, nbr, nA, tag, fc = self._keep
        d = bte_umesh_desc()
        d.dim, d.ncells, d.nfaces = mesh.dim, mesh.ncells, mesh.nfaces
        d.volume = vol.ctypes.data_as(_dp)
        d.owner = own.ctypes.data_as(C.POINTER(C.c_longlong))
        d.neighbor = nbr.ctypes.data_as(C.POINTER(C.c_longlong))
        d.nA = nA.ctypes.data_as(_dp)
        d.tag = tag.ctypes.data_as(_ip)
        d.fc = fc.ctypes.data_as(_dp)
        h = C.c_void_p()
        _ucheck(None, lib().bte_umesh_create(C.byref(d), C.byref(o), C.byref(h)))
        self.h = h
        b = bands
        arrs = [np.ascontiguousarray(x, dtype=np.float64) for x in (b.omega_lo, b.omega_hi, b.vg, b.beta, b.degeneracy)]
        _ucheck(h, lib().bte_umesh_set_bands(h, len(arrs[2]), *(a.ctypes.data_as(_dp) for a in arrs)))
        for t, (kind, T) in bc.items():
            self.set_bc(t, kind, T)
        if T_init is None:
            _ucheck(h, lib().bte_umesh_set_initial(h, None, float(mesh.T_init)))
        else:
            Tc = np.ascontiguousarray(np.broadcast_to(np.asarray(T_init, dtype=np.float64), (mesh.ncells,)))
            _ucheck(h, lib().bte_umesh_set_initial(h, Tc.ctypes.data_as(_dp), 0.0))

    def set_bc(self, tag, kind, T=None):
        """Condition of one boundary tag (as in bc); may be called between steps."""
        if kind in (BTE_BC_ISOTHERMAL, BTE_BC_PARTIAL) and T is not None and not np.isscalar(T):
            Tf = np.ascontiguousarray(T, dtype=np.float64)
            _ucheck(self.h, lib().bte_umesh_set_bc(self.h, int(tag), kind, Tf.ctypes.data_as(_dp), 0.0))
        else:
            _ucheck(self.h, lib().bte_umesh_set_bc(self.h, int(tag), kind, None, float(T) if T is not None else 0.0))

    def step(self, dt, nsteps, ninner, scheme=BTE_IMPLICIT_JACOBI, want_stats=True):
        st = bte_stats() if want_stats else None
        rc = lib().bte_umesh_step(self.h, float(dt), int(nsteps), int(ninner), int(scheme),
                                  C.byref(st) if st is not None else None)
        _ucheck(self.h, rc)
        return rc, (st.as_dict() if st is not None else None)

    def T(self, which=BTE_T_LATTICE):
        out = np.zeros(self.mesh.ncells)
        _ucheck(self.h, lib().bte_umesh_get_T(self.h, which, out.ctypes.data_as(C.c_void_p), 0))
        return out

    def intensity(self):
        out = np.zeros((self.mesh.ncells, self.dirs.nd, len(self.bands.vg)))
        _ucheck(self.h, lib().bte_umesh_get_intensity(self.h, out.ctypes.data_as(_dp)))
        return out

    def set_state(self, I, Tp):
        """Checkpoint restore: intensities [ncells, nd, nb] and T_p [ncells]."""
        I = np.ascontiguousarray(I, dtype=np.float64)
        Tp = np.ascontiguousarray(Tp, dtype=np.float64)
        _ucheck(self.h, lib().bte_umesh_set_intensity(self.h, I.ctypes.data_as(_dp), Tp.ctypes.data_as(_dp)))

    def flux(self):
        q = np.zeros((self.mesh.ncells, 3))
        Q = np.zeros(self.mesh.nfaces)
        _ucheck(self.h, lib().bte_umesh_get_flux(self.h, q.ctypes.data_as(_dp), Q.ctypes.data_as(_dp)))
        return q, Q

    def close(self):
        if getattr(self, "h", None):
            lib().bte_umesh_destroy(self.h)
            self.h = None

    def __del__(self):  # also frees the handle when the constructor failed after bte_umesh_create
        try:
            self.close()
        except Exception:
            pass
