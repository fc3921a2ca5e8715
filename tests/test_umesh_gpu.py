"""Unstructured meshes through the C ABI (bte_umesh_*) against the oracle's
unstructured update.

Bar (FP64): temperatures within rel 1e-12, intensities within rel 1e-11,
cell fluxes within 1e-10 of the largest and boundary-face heat flows within
1e-10 of the largest, on a jittered triangle mesh with 400 directions x 55
bands and all three wall kinds (implicit and explicit), a tetrahedral box,
a mesh read from a Gmsh file, and a quad mesh checked against the
structured handle on the same grid.  A 64x64x2-triangle mesh is checked at
sampled outputs one by one.  Temperature-dependent relaxation rates
(beta_exp) are checked in FP64 (implicit and explicit) and FP32."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O
from paper_2305_19400_gb300 import bte, mesh as M, workloads as W

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2305_19400_gb300 import build as B
    B.build()
    O.build()


def bc_pairs(m, kinds, temps):
    """{tag: (kind, T)} for the solver and the oracle (same constants)."""
    return {t: (k, T) for t, k, T in zip(range(len(kinds)), kinds, temps)}


def run_both(m, dirs, bands, bc, dt, nsteps, ninner, scheme=bte.BTE_IMPLICIT_JACOBI, T_init=None):
    s = bte.UMeshSolver(m, dirs, bands, bc, T_init=T_init)
    rc, st = s.step(dt, nsteps, ninner, scheme)
    assert rc >= 0 and st["nonfinite"] == 0
    u = O.UMeshProblem(m, O.dirs_for(dirs), bands, bc)
    ost = u.init_state(m.T_init if T_init is None else T_init)
    u.run(ost, dt, nsteps, ninner, O.EXPLICIT if scheme == bte.BTE_EXPLICIT else O.IMPLICIT)
    return s, u, ost, st


def assert_matches(s, u, ost):
    for which, key in ((bte.BTE_T_LATTICE, "TL"), (bte.BTE_T_PSEUDO, "Tp")):
        T = s.T(which)
        assert np.max(np.abs(T - ost[key]) / ost[key]) <= 1e-12, key
    I = s.intensity()
    assert np.max(np.abs(I - ost["I"]) / np.abs(ost["I"])) <= 1e-11
    q, Q = s.flux()
    q_ref, Q_ref = u.flux(ost["I"])
    assert np.max(np.abs(q - q_ref)) <= 1e-10 * np.max(np.abs(q_ref))
    assert np.max(np.abs(Q - Q_ref)) <= 1e-10 * max(np.max(np.abs(Q_ref)), 1e-300)


def hot_wall(m, tag, base, amp):
    """Per-face temperatures along a wall: base + amp x (position along y)."""
    T = np.zeros(m.nfaces)
    f = m.boundary_faces(tag)
    y = m.face_center[f, 1]
    T[f] = base + amp * (y - y.min()) / max(np.ptp(y), 1e-300)
    return T


@pytest.mark.parametrize("scheme,dt,nsteps,ninner", [(bte.BTE_IMPLICIT_JACOBI, 1e-12, 3, 5),
                                                     (bte.BTE_EXPLICIT, 2e-13, 12, 1)])
def test_jittered_triangles_400_directions_all_wall_kinds(scheme, dt, nsteps, ninner):
    m = M.tri_grid(13, 9, 130e-9, 90e-9, jitter=0.3, seed=21)
    dirs = W.Dirs("polar_azim", n_polar=20, n_azim=20)
    bands = W.make_bands(40, 15, 19406)
    bc = {0: (bte.BTE_BC_ISOTHERMAL, hot_wall(m, 0, 305.0, 5.0)), 1: (bte.BTE_BC_ISOTHERMAL, 300.0),
          2: (bte.BTE_BC_SPECULAR, None), 3: (bte.BTE_BC_DIFFUSE, None)}
    s, u, ost, st = run_both(m, dirs, bands, bc, dt, nsteps, ninner, scheme)
    assert st["launches"] == nsteps * ninner * 4          # sweep, per-cell step, fix-up, diffuse ghosts
    assert_matches(s, u, ost)
    assert np.max(ost["TL"]) > 300.05                     # heat came in through the hot wall
    s.close()


def test_tetrahedral_box_matches_oracle():
    m = M.tet_box(3, 3, 2, 30e-9, 30e-9, 20e-9)
    dirs = W.Dirs("polar_azim", n_polar=4, n_azim=8)
    bands = W.make_bands(8, 3, 52)
    bc = {0: (bte.BTE_BC_ISOTHERMAL, 306.0), 1: (bte.BTE_BC_ISOTHERMAL, 300.0), 2: (bte.BTE_BC_SPECULAR, None),
          3: (bte.BTE_BC_SPECULAR, None), 4: (bte.BTE_BC_DIFFUSE, None), 5: (bte.BTE_BC_SPECULAR, None)}
    T0 = W.random_temperatures(m.ncells, 23, 299.0, 303.0)
    s, u, ost, _ = run_both(m, dirs, bands, bc, 1e-12, 3, 4, T_init=T0)
    assert_matches(s, u, ost)
    s.close()


def test_mesh_read_from_a_gmsh_file(tmp_path):
    nx, ny, L = 6, 5, 10e-9
    pts = M._grid_points(nx, ny, nx * L, ny * L)
    vid = lambda i, j: j * (nx + 1) + i
    el, bf = [], []
    for j in range(ny):
        for i in range(nx):
            a, b, c, d = vid(i, j), vid(i + 1, j), vid(i + 1, j + 1), vid(i, j + 1)
            el += [("tri", (a, b, c)), ("tri", (a, c, d))] if (i + j) % 3 else [("quad", (a, b, c, d))]
    for j in range(ny):
        bf += [(11, (vid(0, j), vid(0, j + 1))), (12, (vid(nx, j), vid(nx, j + 1)))]
    for i in range(nx):
        bf += [(13, (vid(i, 0), vid(i + 1, 0))), (13, (vid(i, ny), vid(i + 1, ny)))]
    path = str(tmp_path / "mixed.msh")
    M.write_gmsh(path, pts, el, bf)
    m = M.read_gmsh(path)
    assert m.tags == [11, 12, 13]
    dirs = W.Dirs("inplane", n_inplane=16)
    bands = W.make_bands(6, 2, 53)
    bc = {11: (bte.BTE_BC_ISOTHERMAL, 308.0), 12: (bte.BTE_BC_ISOTHERMAL, 300.0), 13: (bte.BTE_BC_SPECULAR, None)}
    s, u, ost, _ = run_both(m, dirs, bands, bc, 1e-12, 4, 5)
    assert_matches(s, u, ost)
    s.close()


def test_quad_mesh_agrees_with_the_structured_handle():
    nx, ny, dx = 11, 7, 10e-9
    wl = W.cfg2(nx, ny)
    g = wl.geoms[0]
    st = bte.Solver(wl)
    st.step(nsteps=3, ninner=5)
    m = M.quad_grid(nx, ny, nx * g.dx, ny * g.dy)
    Th = np.zeros(m.nfaces)
    for f in m.boundary_faces(0):
        Th[f] = g.bc[0][1][int(m.face_center[f, 1] // g.dy)]
    bc = {0: (bte.BTE_BC_ISOTHERMAL, Th), 1: (bte.BTE_BC_ISOTHERMAL, g.bc[1][1][0]),
          2: (bte.BTE_BC_SPECULAR, None), 3: (bte.BTE_BC_SPECULAR, None)}
    s = bte.UMeshSolver(m, wl.dirs, wl.bands, bc, T_init=g.T_init)
    s.step(wl.dt, 3, 5)
    assert np.max(np.abs(s.T(bte.BTE_T_LATTICE) - st.T(0, bte.BTE_T_LATTICE)) / 300.0) <= 1e-13
    assert np.max(np.abs(s.intensity() - st.intensity(0)) / st.intensity(0)) <= 1e-12
    s.close()
    st.close()


def test_argument_and_order_errors():
    m = M.tri_grid(4, 3, 40e-9, 30e-9, jitter=0.2, seed=2)
    dirs = W.Dirs("inplane", n_inplane=8)
    bands = W.make_bands(3, 1, 54)
    with pytest.raises(bte.BTEError) as e:      # a mirror needs axis-normal faces: turn the mesh by 30 degrees
        pts_turned = M.tri_grid(4, 3, 40e-9, 30e-9)
        c, s_ = np.cos(0.5236), np.sin(0.5236)
        R = np.array([[c, -s_, 0], [s_, c, 0], [0, 0, 1]])
        mt = M.UMesh(2, pts_turned.volume, pts_turned.owner, pts_turned.neighbor, pts_turned.nA @ R.T,
                     pts_turned.tag, pts_turned.centroid @ R.T, pts_turned.face_center @ R.T)
        bte.UMeshSolver(mt, dirs, bands, {0: (bte.BTE_BC_SPECULAR, None), 1: (0, 300.0), 2: (0, 300.0), 3: (0, 300.0)})
    assert e.value.code == -1
    with pytest.raises(bte.BTEError) as e:      # so does a partially specular tag
        bte.UMeshSolver(mt, dirs, bands, {0: (bte.BTE_BC_PARTIAL, 0.5), 1: (0, 300.0), 2: (0, 300.0), 3: (0, 300.0)})
    assert e.value.code == -1
    with pytest.raises(bte.BTEError) as e:      # an unknown tag
        bte.UMeshSolver(m, dirs, bands, {7: (bte.BTE_BC_SPECULAR, None)})
    assert e.value.code == -1
    s = bte.UMeshSolver(m, dirs, bands, {0: (0, 305.0), 1: (0, 300.0), 2: (1, None)})  # tag 3 left out
    with pytest.raises(bte.BTEError) as e:
        s.step(1e-12, 1, 1)
    assert e.value.code == -2
    s.close()


def test_sampled_outputs_on_a_64x64x2_triangle_mesh():
    m = M.tri_grid(64, 64, 640e-9, 640e-9, jitter=0.25, seed=31)
    dirs = W.Dirs("polar_azim", n_polar=20, n_azim=20)
    bands = W.make_bands(40, 15, 19406)
    bc = {0: (bte.BTE_BC_ISOTHERMAL, hot_wall(m, 0, 305.0, 10.0)), 1: (bte.BTE_BC_ISOTHERMAL, 300.0),
          2: (bte.BTE_BC_SPECULAR, None), 3: (bte.BTE_BC_DIFFUSE, None)}
    s = bte.UMeshSolver(m, dirs, bands, bc)
    s.step(1e-12, 1, 3)
    I_n = s.intensity()
    Tp_n = s.T(bte.BTE_T_PSEUDO)
    s.step(1e-12, 1, 1)
    I_1 = s.intensity()
    Tp_1, TL_1 = s.T(bte.BTE_T_PSEUDO), s.T(bte.BTE_T_LATTICE)
    u = O.UMeshProblem(m, O.dirs_for(dirs), bands, bc)
    I0w = u.wall_I0()
    rng = np.random.default_rng(4)
    nc, nd, nb = I_n.shape
    cells = set(rng.integers(0, nc, 30).tolist()) | set(int(m.owner[f]) for f in m.boundary_faces()[::17])
    I0 = np.zeros((nc, nb))
    for P in cells:
        I0[P] = O.I0(bands, Tp_n[P])[0]
    # the diffuse ghosts of the pass come from I^n (the step's first iterate)
    worst = 0.0
    for P in sorted(cells):
        for d in rng.integers(0, nd, 8):
            for b in rng.integers(0, nb, 4):
                ref = u.update_one(1e-12, O.IMPLICIT, I_n, I_n, I0, I0w, P, d, b)
                worst = max(worst, abs(I_1[P, d, b] - ref) / abs(ref))
        Tp_ref, TL_ref = u.tables.cell_temperatures(I_1[P], Tp_n[P], Tp_n[P])
        assert abs(Tp_1[P] - Tp_ref) <= 1e-12 * Tp_ref
        assert abs(TL_1[P] - TL_ref) <= 1e-12 * TL_ref
    assert worst <= 1e-12, worst
    s.close()


def test_single_triangle_and_one_band():
    pts = np.array([[0.0, 0.0, 0.0], [10e-9, 0.0, 0.0], [0.0, 10e-9, 0.0]])
    m = M.from_elements(pts, [("tri", (0, 1, 2))], {frozenset((0, 1)): 0, frozenset((0, 2)): 1, frozenset((1, 2)): 2})
    bands = W.make_bands(1, 0, 62)
    bc = {0: (bte.BTE_BC_ISOTHERMAL, 310.0), 1: (bte.BTE_BC_SPECULAR, None), 2: (bte.BTE_BC_DIFFUSE, None)}
    s, u, ost, _ = run_both(m, W.Dirs("inplane", n_inplane=12), bands, bc, 1e-12, 5, 4)
    assert_matches(s, u, ost)
    s.close()


def test_hexahedral_gmsh_mesh(tmp_path):
    nx, ny, nz, L = 3, 2, 2, 10e-9
    x, y, z = np.arange(nx + 1) * L, np.arange(ny + 1) * L, np.arange(nz + 1) * L
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    pts = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
    vid = lambda i, j, k: (k * (ny + 1) + j) * (nx + 1) + i
    el, bf = [], []
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                el.append(("hex", (vid(i, j, k), vid(i + 1, j, k), vid(i + 1, j + 1, k), vid(i, j + 1, k),
                                   vid(i, j, k + 1), vid(i + 1, j, k + 1), vid(i + 1, j + 1, k + 1), vid(i, j + 1, k + 1))))
    for k in range(nz):
        for j in range(ny):
            bf.append((1, (vid(0, j, k), vid(0, j + 1, k), vid(0, j + 1, k + 1), vid(0, j, k + 1))))
            bf.append((2, (vid(nx, j, k), vid(nx, j + 1, k), vid(nx, j + 1, k + 1), vid(nx, j, k + 1))))
    path = str(tmp_path / "hex.msh")
    M.write_gmsh(path, pts, el, bf)
    m = M.read_gmsh(path)           # y and z sides are untagged: default tag 0
    assert m.tags == [0, 1, 2] and m.closure_residual() < 1e-14
    bc = {0: (bte.BTE_BC_SPECULAR, None), 1: (bte.BTE_BC_ISOTHERMAL, 307.0), 2: (bte.BTE_BC_ISOTHERMAL, 300.0)}
    s, u, ost, _ = run_both(m, W.Dirs("polar_azim", n_polar=4, n_azim=8), W.make_bands(6, 2, 63), bc, 1e-12, 3, 4)
    assert_matches(s, u, ost)
    s.close()


@pytest.mark.parametrize("precision,tol,scheme,dt,nsteps,ninner", [
    (bte.BTE_FP32, 1e-4, bte.BTE_IMPLICIT_JACOBI, 1e-12, 3, 8),
    (bte.BTE_FP32, 1e-4, bte.BTE_EXPLICIT, 2e-13, 12, 1),
    (bte.BTE_BF16, 2e-3, bte.BTE_IMPLICIT_JACOBI, 1e-12, 3, 8)])
def test_reduced_storage_on_jittered_triangles(precision, tol, scheme, dt, nsteps, ninner):
    """FP32 (BF16) deviation storage against the FP64 oracle: max |dT| within
    1e-4 K (2e-3 K for BF16, short runs only) on the 400-direction mesh with
    every wall kind; heat flux within the same relative bound x 100."""
    m = M.tri_grid(13, 9, 130e-9, 90e-9, jitter=0.3, seed=21)
    dirs = W.Dirs("polar_azim", n_polar=20, n_azim=20)
    bands = W.make_bands(40, 15, 19406)
    bc = {0: (bte.BTE_BC_ISOTHERMAL, hot_wall(m, 0, 305.0, 5.0)), 1: (bte.BTE_BC_ISOTHERMAL, 300.0),
          2: (bte.BTE_BC_SPECULAR, None), 3: (bte.BTE_BC_DIFFUSE, None)}
    s = bte.UMeshSolver(m, dirs, bands, bc, precision=precision)
    rc, st = s.step(dt, nsteps, ninner, scheme)
    assert rc >= 0 and st["nonfinite"] == 0
    u = O.UMeshProblem(m, O.dirs_for(dirs), bands, bc)
    ost = u.init_state(m.T_init)
    u.run(ost, dt, nsteps, ninner, O.EXPLICIT if scheme == bte.BTE_EXPLICIT else O.IMPLICIT)
    assert np.max(np.abs(s.T(bte.BTE_T_LATTICE) - ost["TL"])) <= tol
    assert np.max(np.abs(s.T(bte.BTE_T_PSEUDO) - ost["Tp"])) <= tol
    q, Q = s.flux()
    q_ref, Q_ref = u.flux(ost["I"])
    assert np.linalg.norm(q - q_ref) <= 100 * tol * np.linalg.norm(q_ref)
    assert np.max(np.abs(Q - Q_ref)) <= 100 * tol * np.max(np.abs(Q_ref))
    I = s.intensity()
    assert np.max(np.abs(I - ost["I"]) / np.abs(ost["I"])) <= 100 * tol
    s.close()


def test_fp32_tetrahedra_with_diffuse_walls():
    m = M.tet_box(3, 3, 2, 30e-9, 30e-9, 20e-9)
    bc = {0: (bte.BTE_BC_ISOTHERMAL, 306.0), 1: (bte.BTE_BC_ISOTHERMAL, 300.0), 2: (bte.BTE_BC_DIFFUSE, None),
          3: (bte.BTE_BC_SPECULAR, None), 4: (bte.BTE_BC_DIFFUSE, None), 5: (bte.BTE_BC_SPECULAR, None)}
    dirs = W.Dirs("polar_azim", n_polar=4, n_azim=8)
    bands = W.make_bands(8, 3, 52)
    s = bte.UMeshSolver(m, dirs, bands, bc, precision=bte.BTE_FP32)
    s.step(1e-12, 3, 4)
    u = O.UMeshProblem(m, O.dirs_for(dirs), bands, bc)
    ost = u.init_state(m.T_init)
    u.run(ost, 1e-12, 3, 4)
    assert np.max(np.abs(s.T(bte.BTE_T_LATTICE) - ost["TL"])) <= 1e-4
    s.close()


@pytest.mark.parametrize("precision", [bte.BTE_FP64, bte.BTE_FP32])
def test_checkpoint_restore_continues_the_run(precision):
    m = M.tri_grid(9, 7, 90e-9, 70e-9, jitter=0.2, seed=41)
    dirs = W.Dirs("inplane", n_inplane=16)
    bands = W.make_bands(6, 2, 64)
    bc = {0: (bte.BTE_BC_ISOTHERMAL, 309.0), 1: (bte.BTE_BC_ISOTHERMAL, 300.0), 2: (bte.BTE_BC_SPECULAR, None),
          3: (bte.BTE_BC_DIFFUSE, None)}
    a = bte.UMeshSolver(m, dirs, bands, bc, precision=precision)
    a.step(1e-12, 3, 5)
    I, Tp = a.intensity(), a.T(bte.BTE_T_PSEUDO)
    a.step(1e-12, 2, 5)
    b = bte.UMeshSolver(m, dirs, bands, bc, precision=precision)
    b.set_state(I, Tp)
    b.step(1e-12, 2, 5)
    # the restore evaluates I0 exactly at T_p where the run carried its cached model: round-off apart
    tol_T, tol_I = (1e-14, 1e-13) if precision == bte.BTE_FP64 else (1e-12, 1e-6)
    assert np.max(np.abs(b.T(bte.BTE_T_LATTICE) - a.T(bte.BTE_T_LATTICE)) / a.T(bte.BTE_T_LATTICE)) <= tol_T
    assert np.max(np.abs(b.intensity() - a.intensity()) / a.intensity()) <= tol_I
    a.close()
    b.close()


@pytest.mark.parametrize("precision,scheme,dt,nsteps,ninner", [
    (bte.BTE_FP64, bte.BTE_IMPLICIT_JACOBI, 1e-12, 3, 5),
    (bte.BTE_FP64, bte.BTE_EXPLICIT, 2e-13, 12, 1),
    (bte.BTE_FP32, bte.BTE_IMPLICIT_JACOBI, 1e-12, 3, 5)])
def test_temperature_dependent_relaxation_on_jittered_triangles(precision, scheme, dt, nsteps, ninner):
    """beta_b(T_p) = beta_b (T_p / 300 K)^-1.2 per cell against the oracle: FP64
    within rel 1e-12 on T and 1e-11 on I, FP32 within 1e-4 K."""
    m = M.tri_grid(13, 9, 130e-9, 90e-9, jitter=0.3, seed=25)
    dirs = W.Dirs("polar_azim", n_polar=20, n_azim=20)
    bands = W.make_bands(40, 15, 19408)
    bc = {0: (bte.BTE_BC_ISOTHERMAL, hot_wall(m, 0, 320.0, 10.0)), 1: (bte.BTE_BC_ISOTHERMAL, 300.0),
          2: (bte.BTE_BC_SPECULAR, None), 3: (bte.BTE_BC_DIFFUSE, None)}
    s = bte.UMeshSolver(m, dirs, bands, bc, precision=precision, beta_exp=-1.2)
    rc, st = s.step(dt, nsteps, ninner, scheme)
    assert rc >= 0 and st["nonfinite"] == 0
    assert st["launches"] == nsteps * ninner * 5     # + the relaxation scale before every sweep
    u = O.UMeshProblem(m, O.dirs_for(dirs), bands, bc, beta_exp=-1.2, beta_Tref=300.0)
    ost = u.init_state(m.T_init)
    u.run(ost, dt, nsteps, ninner, O.EXPLICIT if scheme == bte.BTE_EXPLICIT else O.IMPLICIT)
    assert np.max(ost["TL"]) > 300.5                   # the hot wall moved the cells' rates
    if precision == bte.BTE_FP64:
        assert_matches(s, u, ost)
    else:
        assert np.max(np.abs(s.T(bte.BTE_T_LATTICE) - ost["TL"])) <= 1e-4
        assert np.max(np.abs(s.T(bte.BTE_T_PSEUDO) - ost["Tp"])) <= 1e-4
    s.close()


def test_relaxation_exponent_out_of_range_is_refused():
    m = M.tri_grid(3, 2, 30e-9, 20e-9)
    with pytest.raises(bte.BTEError) as e:
        bte.UMeshSolver(m, W.Dirs("inplane", n_inplane=8), W.make_bands(2, 0, 3),
                        {t: (bte.BTE_BC_SPECULAR, None) for t in range(4)}, beta_exp=20.0)
    assert e.value.code == -1
