"""Axisymmetric problems on the GPU: one wedge of a hollow cylinder about the
z axis (mesh.wedge_ring) whose two side faces take BTE_BC_ROTATIONAL, with
the paper's 20 x 20 direction set (wedge angle 18 degrees, one azimuthal
bin) and 55 band-polarisations.

* FP64, implicit and explicit: temperatures within rel 1e-12 of the oracle's
  wedge, intensities within rel 1e-11, boundary-face heat flows within 1e-10
  of the largest (the oracle's rotational faces are pinned against the full
  ring of wedges on the CPU);
* the GPU wedge against the GPU's own full ring of 20 wedges (no rotational
  faces): the same temperatures in every wedge, and the intensities of wedge
  k equal to the wedge's after rotating the directions by k bins;
* FP32 deviation storage within 1e-4 K of the oracle;
* refused: an angle the direction set does not map onto itself, two tags
  with different angles, a negative or non-finite angle, a mesh without face
  centres, a face that is no plane through the axis."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O
from paper_2305_19400_gb300 import bte, mesh as M, workloads as W

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

NPHI = 20
ALPHA = 2 * np.pi / NPHI
DIRS = W.Dirs("polar_azim", n_polar=20, n_azim=NPHI)


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2305_19400_gb300 import build as B
    B.build()
    O.build()


def _walls(rot=True):
    bc = {0: (bte.BTE_BC_ISOTHERMAL, 312.0), 1: (bte.BTE_BC_ISOTHERMAL, 300.0), 2: (bte.BTE_BC_SPECULAR, None),
          3: (bte.BTE_BC_DIFFUSE, None)}
    if rot:
        bc.update({4: (bte.BTE_BC_ROTATIONAL, ALPHA), 5: (bte.BTE_BC_ROTATIONAL, ALPHA)})
    return bc


def _wedge(nwedge=1):
    return M.wedge_ring(5, 6, 30e-9, 130e-9, 60e-9, ALPHA, nwedge=nwedge)


@pytest.mark.parametrize("scheme,dt,nsteps,ninner", [(bte.BTE_IMPLICIT_JACOBI, 1e-12, 3, 5),
                                                     (bte.BTE_EXPLICIT, 2e-13, 12, 1)])
def test_fp64_wedge_matches_the_oracle(scheme, dt, nsteps, ninner):
    m = _wedge()
    bands = W.make_bands(40, 15, 19407)
    s = bte.UMeshSolver(m, DIRS, bands, _walls())
    rc, st = s.step(dt, nsteps, ninner, scheme)
    assert rc >= 0 and st["nonfinite"] == 0
    u = O.UMeshProblem(m, O.dirs_for(DIRS), bands, _walls())
    ost = u.init_state(m.T_init)
    u.run(ost, dt, nsteps, ninner, O.EXPLICIT if scheme == bte.BTE_EXPLICIT else O.IMPLICIT)
    for which, key in ((bte.BTE_T_LATTICE, "TL"), (bte.BTE_T_PSEUDO, "Tp")):
        assert np.max(np.abs(s.T(which) - ost[key]) / ost[key]) <= 1e-12, key
    I = s.intensity()
    assert np.max(np.abs(I - ost["I"]) / np.abs(ost["I"])) <= 1e-11
    _, Q = s.flux()
    _, Q_ref = u.flux(ost["I"])
    assert np.max(np.abs(Q - Q_ref)) <= 1e-10 * np.max(np.abs(Q_ref))
    side = np.concatenate([m.boundary_faces(4), m.boundary_faces(5)])
    # the two sides of a wedge pass the same energy per unit time: their net flows cancel
    assert abs(Q[m.boundary_faces(4)].sum() + Q[m.boundary_faces(5)].sum()) <= 1e-10 * np.max(np.abs(Q_ref))
    assert np.max(ost["TL"]) > 300.05 and side.size == 2 * 5 * 6
    s.close()


def test_gpu_wedge_equals_the_gpu_full_ring():
    bands = W.make_bands(12, 4, 19408)
    w, ring = _wedge(), _wedge(NPHI)
    a = bte.UMeshSolver(w, DIRS, bands, _walls())
    b = bte.UMeshSolver(ring, DIRS, bands, _walls(rot=False))
    for s in (a, b):
        s.step(1e-12, 2, 6)
    Tw, Tr = a.T(bte.BTE_T_LATTICE), b.T(bte.BTE_T_LATTICE)
    Iw, Ir = a.intensity(), b.intensity()
    nc, ntheta = w.ncells, DIRS.n_polar
    for k in range(NPHI):
        assert np.max(np.abs(Tr[k * nc:(k + 1) * nc] - Tw) / Tw) <= 1e-12
        rot = np.array([i * NPHI + (j - k) % NPHI for i in range(ntheta) for j in range(NPHI)])
        Ik = Ir[k * nc:(k + 1) * nc]
        assert np.max(np.abs(Ik - Iw[:, rot, :]) / np.abs(Ik)) <= 1e-11
    a.close()
    b.close()


def test_fp32_wedge_within_the_reduced_mode_bar():
    m = _wedge()
    bands = W.make_bands(40, 15, 19407)
    s = bte.UMeshSolver(m, DIRS, bands, _walls(), precision=bte.BTE_FP32)
    s.step(1e-12, 3, 5)
    u = O.UMeshProblem(m, O.dirs_for(DIRS), bands, _walls())
    ost = u.init_state(m.T_init)
    u.run(ost, 1e-12, 3, 5)
    assert np.max(np.abs(s.T(bte.BTE_T_LATTICE) - ost["TL"])) <= 1e-4
    assert np.max(np.abs(s.T(bte.BTE_T_PSEUDO) - ost["Tp"])) <= 1e-4
    s.close()


def test_rotational_faces_refuse_what_they_cannot_represent():
    m = _wedge()
    bands = W.make_bands(4, 1, 19409)
    walls = {k: v for k, v in _walls().items() if k < 4}
    s = bte.UMeshSolver(m, DIRS, bands, {**walls, 4: (bte.BTE_BC_ROTATIONAL, ALPHA), 5: (bte.BTE_BC_ROTATIONAL, ALPHA)})
    for tag, angle in ((4, 2 * np.pi / 7), (5, 2 * ALPHA), (4, -ALPHA), (4, float("nan"))):
        with pytest.raises(bte.BTEError) as e:
            s.set_bc(tag, bte.BTE_BC_ROTATIONAL, angle)
        assert e.value.code == bte.BTE_E_ARG
    with pytest.raises(bte.BTEError):           # the outer surface is no plane through the axis
        s.set_bc(1, bte.BTE_BC_ROTATIONAL, ALPHA)
    s.step(1e-12, 1, 2)                          # the handle still steps with its valid conditions
    assert np.all(np.isfinite(s.T(bte.BTE_T_LATTICE)))
    s.close()
    with pytest.raises(bte.BTEError) as e:      # no rotation of the 20 x 20 set by 2 pi / 7
        bte.UMeshSolver(m, DIRS, bands, {**walls, 4: (bte.BTE_BC_ROTATIONAL, 2 * np.pi / 7),
                                         5: (bte.BTE_BC_ROTATIONAL, 2 * np.pi / 7)})
    assert e.value.code == bte.BTE_E_ARG and "direction set" in str(e.value)


def test_a_mesh_without_face_centres_cannot_take_rotational_faces():
    import ctypes as C
    m = _wedge()
    L = bte.lib()
    keep = [np.ascontiguousarray(m.volume), np.ascontiguousarray(m.owner, dtype=np.int64),
            np.ascontiguousarray(m.neighbor, dtype=np.int64), np.ascontiguousarray(m.nA),
            np.ascontiguousarray(m.tag, dtype=np.int32)]
    d = bte.bte_umesh_desc()
    d.dim, d.ncells, d.nfaces = 3, m.ncells, m.nfaces
    d.volume = keep[0].ctypes.data_as(C.POINTER(C.c_double))
    d.owner = keep[1].ctypes.data_as(C.POINTER(C.c_longlong))
    d.neighbor = keep[2].ctypes.data_as(C.POINTER(C.c_longlong))
    d.nA = keep[3].ctypes.data_as(C.POINTER(C.c_double))
    d.tag = keep[4].ctypes.data_as(C.POINTER(C.c_int))   # fc left NULL
    o = bte.bte_default_opts()
    o.dir_kind, o.n_polar, o.n_azim = bte.BTE_DIRS_POLAR_AZIM, 4, NPHI
    o.cuda_stream = torch.cuda.current_stream().cuda_stream
    h = C.c_void_p()
    assert L.bte_umesh_create(C.byref(d), C.byref(o), C.byref(h)) == 0
    b = W.make_bands(2, 0, 3)
    arrs = [np.ascontiguousarray(x, dtype=np.float64) for x in (b.omega_lo, b.omega_hi, b.vg, b.beta, b.degeneracy)]
    assert L.bte_umesh_set_bands(h, 2, *(x.ctypes.data_as(C.POINTER(C.c_double)) for x in arrs)) == 0
    assert L.bte_umesh_set_bc(h, 4, bte.BTE_BC_ROTATIONAL, None, ALPHA) == bte.BTE_E_ARG
    assert b"face centres" in L.bte_umesh_last_error(h)
    L.bte_umesh_destroy(h)
