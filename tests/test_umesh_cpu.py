"""Unstructured meshes on the CPU: the face-list builder and the Gmsh / MEDIT
readers, and the oracle's unstructured update pinned against facts that do
not come from it: the structured oracle on the same grid (a quad mesh is the
structured grid), a dense LU solve of the backward-Euler system assembled
here from the face data, equilibrium, energy conservation in closed
enclosures, and invariance under a 90-degree rotation of the mesh."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2305_19400_gb300 import mesh as M, workloads as W


# ------------------------------------------------------------------- meshes
@pytest.mark.parametrize("mk", [lambda: M.quad_grid(5, 4, 50e-9, 40e-9),
                                lambda: M.tri_grid(6, 5, 60e-9, 50e-9, jitter=0.3, seed=1),
                                lambda: M.tet_box(3, 2, 2, 30e-9, 20e-9, 20e-9)])
def test_face_lists_close_every_cell_and_tile_the_domain(mk):
    m = mk()
    assert m.closure_residual() < 1e-14
    size = {2: (50e-9 * 40e-9, 60e-9 * 50e-9), 3: (30e-9 * 20e-9 * 20e-9,)}
    assert any(abs(m.volume.sum() - v) < 1e-12 * v for v in size[m.dim])
    # each boundary tag's area vectors add up to the side's outward area
    for t in m.tags:
        f = m.boundary_faces(t)
        tot = m.nA[f].sum(axis=0)
        assert abs(np.linalg.norm(tot) - np.linalg.norm(m.nA[f], axis=1).sum()) < 1e-12 * np.linalg.norm(tot)
    # outward: from the owner's centroid towards the face
    assert np.all(np.einsum("ij,ij->i", m.face_center - m.centroid[m.owner], m.nA) > 0)


def _elements_of_tri_grid(nx, ny, Lx, Ly):
    pts = M._grid_points(nx, ny, Lx, Ly)
    vid = lambda i, j: j * (nx + 1) + i
    el, bf = [], []
    for j in range(ny):
        for i in range(nx):
            a, b, c, d = vid(i, j), vid(i + 1, j), vid(i + 1, j + 1), vid(i, j + 1)
            el += [("tri", (a, b, c)), ("tri", (a, c, d))]
    for j in range(ny):
        bf += [(7, (vid(0, j), vid(0, j + 1))), (8, (vid(nx, j), vid(nx, j + 1)))]
    for i in range(nx):
        bf += [(9, (vid(i, 0), vid(i + 1, 0))), (10, (vid(i, ny), vid(i + 1, ny)))]
    return pts, el, bf


@pytest.mark.parametrize("fmt", ["gmsh", "medit"])
def test_mesh_files_read_back_to_the_same_face_list(tmp_path, fmt):
    pts, el, bf = _elements_of_tri_grid(4, 3, 40e-9, 30e-9)
    ref = M.from_elements(pts, el, {frozenset(v): t for t, v in bf})
    path = str(tmp_path / ("m.msh" if fmt == "gmsh" else "m.mesh"))
    if fmt == "gmsh":
        M.write_gmsh(path, pts, el, bf)
        m = M.read_gmsh(path)
    else:
        M.write_medit(path, pts, el, bf, 2)
        m = M.read_medit(path)
    assert m.dim == 2 and m.ncells == ref.ncells and m.nfaces == ref.nfaces
    assert np.allclose(m.volume, ref.volume, rtol=1e-15, atol=0)
    assert np.array_equal(m.owner, ref.owner) and np.array_equal(m.neighbor, ref.neighbor)
    assert np.allclose(m.nA, ref.nA, rtol=0, atol=1e-24)
    assert np.array_equal(m.tag, ref.tag) and m.tags == [7, 8, 9, 10]


def test_tetrahedral_gmsh_file_reads(tmp_path):
    b = M.tet_box(2, 2, 1, 20e-9, 20e-9, 10e-9)
    # rebuild the same elements through a file: write the box's tets and its tagged facets
    pts, el, bf = _tet_box_elements(2, 2, 1, 20e-9, 20e-9, 10e-9)
    path = str(tmp_path / "box.msh")
    M.write_gmsh(path, pts, el, bf)
    m = M.read_gmsh(path)
    assert m.dim == 3 and m.ncells == b.ncells and abs(m.volume.sum() - b.volume.sum()) < 1e-12 * b.volume.sum()
    assert m.tags == [0, 1, 2, 3, 4, 5] and m.closure_residual() < 1e-14


def _tet_box_elements(nx, ny, nz, Lx, Ly, Lz):
    x, y, z = np.linspace(0, Lx, nx + 1), np.linspace(0, Ly, ny + 1), np.linspace(0, Lz, nz + 1)
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    pts = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
    vid = lambda i, j, k: (k * (ny + 1) + j) * (nx + 1) + i
    el, bf = [], []
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                c = [vid(i + a, j + b, k + e) for e in (0, 1) for b in (0, 1) for a in (0, 1)]
                for p, q in ((1, 3), (3, 2), (2, 6), (6, 4), (4, 5), (5, 1)):
                    tet = (c[0], c[p], c[q], c[7])
                    el.append(("tet", tet))
                    for fac in ((0, 1, 2), (0, 1, 3), (0, 2, 3), (1, 2, 3)):
                        v = [tet[s] for s in fac]
                        P = pts[v]
                        for ax, lo, hi, t0 in ((0, 0, Lx, 0), (1, 0, Ly, 2), (2, 0, Lz, 4)):
                            if np.all(P[:, ax] == lo): bf.append((t0, tuple(v)))
                            if np.all(P[:, ax] == hi): bf.append((t0 + 1, tuple(v)))
    return pts, el, bf


# ------------------------------------------------------------ oracle pins
def _mixed_rectangle(nx, ny, dx, walls=((W.BC_SPECULAR, None), (W.BC_DIFFUSE, None))):
    """A rectangle with isothermal x sides and the given y sides, as a structured
    grid and as a quad mesh with the same walls (tags 0-3 = sides -x, +x, -y, +y)."""
    g = W.Geometry(2, nx, ny, 1, dx, dx, dx)
    Th = W.random_temperatures(ny, 3, 300.0, 310.0)
    g.bc = [(W.BC_ISOTHERMAL, Th), (W.BC_ISOTHERMAL, np.full(ny, 300.0))] + list(walls)
    m = M.quad_grid(nx, ny, nx * dx, ny * dx)
    Twall = np.zeros(m.nfaces)
    for f in m.boundary_faces(0):
        Twall[f] = Th[int(m.face_center[f, 1] // dx)]
    bc = {0: (O.ISOTHERMAL, Twall), 1: (O.ISOTHERMAL, 300.0), 2: walls[0], 3: walls[1]}
    return g, m, bc


@pytest.mark.parametrize("walls", [((W.BC_SPECULAR, None), (W.BC_DIFFUSE, None)),
                                   ((W.BC_PARTIAL, 0.3), (W.BC_PARTIAL, 0.8))])
@pytest.mark.parametrize("scheme,dt,nsteps,ninner", [(O.IMPLICIT, 1e-12, 3, 5), (O.EXPLICIT, 2e-13, 20, 1)])
def test_quad_mesh_reproduces_the_structured_oracle(scheme, dt, nsteps, ninner, walls):
    g, m, bc = _mixed_rectangle(6, 5, 10e-9, walls)
    dirs, bands = O.dirs_inplane(16), W.make_bands(6, 2, 5)
    T0 = W.random_temperatures(30, 4, 298.0, 304.0)
    p = O.Problem(g, dirs, bands)
    st = p.init_state(T0)
    p.run(st, dt, nsteps, ninner, scheme)
    u = O.UMeshProblem(m, dirs, bands, bc)
    su = u.init_state(T0)
    u.run(su, dt, nsteps, ninner, scheme)
    assert np.max(np.abs(su["TL"] - st["TL"]) / st["TL"]) < 1e-14
    assert np.max(np.abs(su["Tp"] - st["Tp"]) / st["Tp"]) < 1e-14
    assert np.max(np.abs(su["I"] - st["I"]) / st["I"]) < 1e-13


@pytest.mark.parametrize("scheme,dt,nsteps,ninner", [(O.IMPLICIT, 1e-12, 3, 5), (O.EXPLICIT, 2e-13, 15, 1)])
def test_quad_mesh_with_temperature_dependent_tau_reproduces_the_structured_oracle(scheme, dt, nsteps, ninner):
    g, m, bc = _mixed_rectangle(6, 5, 10e-9, ((W.BC_PARTIAL, 0.4), (W.BC_DIFFUSE, None)))
    dirs, bands = O.dirs_inplane(16), W.make_bands(6, 2, 5)
    T0 = W.random_temperatures(30, 4, 290.0, 330.0)
    p = O.Problem(g, dirs, bands, beta_exp=-1.5, beta_Tref=300.0)
    st = p.init_state(T0)
    p.run(st, dt, nsteps, ninner, scheme)
    u = O.UMeshProblem(m, dirs, bands, bc, beta_exp=-1.5, beta_Tref=300.0)
    su = u.init_state(T0)
    u.run(su, dt, nsteps, ninner, scheme)
    assert np.max(np.abs(su["TL"] - st["TL"]) / st["TL"]) < 1e-14
    assert np.max(np.abs(su["I"] - st["I"]) / st["I"]) < 1e-13
    fixed = O.UMeshProblem(m, dirs, bands, bc)   # and tau(T) does change the answer
    sf = fixed.init_state(T0)
    fixed.run(sf, dt, nsteps, ninner, scheme)
    assert np.max(np.abs(sf["TL"] - su["TL"])) > 1e-6


def _assemble_unstructured(m, S, w, bands, dt, In, I0w_face):
    """Dense backward-Euler system (beta = 0) from the face list: for each
    (P, d, b), (1/dt) I_P + (v/V_P) sum_f (S_d.n_f A_f / w_d) I_f = I^n_P/dt,
    I_f the upwind value (own for outflow, neighbour or wall ghost inflow)."""
    nc, nd, nb = m.ncells, len(w), len(bands.vg)
    idx = lambda P, d, b: (P * nd + d) * nb + b
    A = np.zeros((nc * nd * nb,) * 2)
    rhs = np.zeros(nc * nd * nb)
    for P in range(nc):
        for d in range(nd):
            for b in range(nb):
                r = idx(P, d, b)
                A[r, r] += 1 / dt
                rhs[r] += In[P, d, b] / dt
    for f in range(m.nfaces):
        for side, P, Q, sgn in ((0, m.owner[f], m.neighbor[f], 1.0), (1, m.neighbor[f], m.owner[f], -1.0)):
            if P < 0:
                continue
            for d in range(nd):
                sn = sgn * float(S[d] @ m.nA[f]) / w[d]
                for b in range(nb):
                    c = bands.vg[b] * sn / m.volume[P]
                    r = idx(P, d, b)
                    if sn > 0:
                        A[r, r] += c
                    elif Q >= 0:
                        A[r, idx(Q, d, b)] += c
                    else:
                        rhs[r] -= c * I0w_face[f][b]
    return A, rhs


def test_jacobi_on_a_triangle_mesh_converges_to_dense_lu_solution():
    m = M.tri_grid(3, 2, 30e-9, 20e-9, jitter=0.25, seed=3)
    S, w, r = O.dirs_inplane(8)
    bands = W.make_bands(2, 0, 7)
    bands.beta[:] = 0.0
    Tw = {0: 310.0, 1: 300.0, 2: 305.0, 3: 295.0}
    u = O.UMeshProblem(m, (S, w, r), bands, {t: (O.ISOTHERMAL, T) for t, T in Tw.items()})
    st = u.init_state(W.random_temperatures(m.ncells, 9, 296.0, 306.0))
    I0w = {f: O.I0(bands, Tw[int(m.tag[f])])[0] for f in m.boundary_faces()}
    dt = 2e-12
    A, rhs = _assemble_unstructured(m, S, w, bands, dt, st["I"].copy(), I0w)
    x = np.linalg.solve(A, rhs).reshape(st["I"].shape)
    u.run(st, dt, 1, 400)
    assert np.max(np.abs(st["I"] - x) / np.abs(x)) < 1e-13


@pytest.mark.parametrize("kinds", [(O.SPECULAR,) * 4, (O.DIFFUSE, O.SPECULAR, O.DIFFUSE, O.DIFFUSE)])
def test_uniform_equilibrium_on_a_jittered_triangle_mesh_stays_at_round_off(kinds):
    m = M.tri_grid(5, 4, 50e-9, 40e-9, jitter=0.3, seed=5)
    bands = W.make_bands(5, 2, 8)
    u = O.UMeshProblem(m, O.dirs_inplane(12), bands, {t: (k, None) for t, k in enumerate(kinds)})
    st = u.init_state(300.0)
    I_init = st["I"].copy()
    u.run(st, 1e-12, 5, 4)
    assert np.max(np.abs(st["I"] - I_init) / I_init) < 1e-13
    assert np.max(np.abs(st["TL"] - 300.0)) < 1e-12


@pytest.mark.parametrize("kind", [O.SPECULAR, O.DIFFUSE, O.PARTIAL])
def test_closed_triangle_enclosure_conserves_energy(kind):
    m = M.tri_grid(6, 5, 60e-9, 50e-9, jitter=0.3, seed=6)
    bands = W.make_bands(4, 1, 9)
    u = O.UMeshProblem(m, O.dirs_inplane(12), bands, {t: (kind, 0.25 + 0.2 * t if kind == O.PARTIAL else None)
                                                       for t in range(4)})
    st = u.init_state(W.random_temperatures(m.ncells, 10, 290.0, 310.0))

    def total(I):
        return sum(m.volume[P] * u.cell_energy(I[P])[0] for P in range(m.ncells))
    E0 = total(st["I"])
    T0 = st["TL"].copy()
    u.run(st, 2e-13, 60, 1, O.EXPLICIT)
    assert abs(total(st["I"]) - E0) <= 1e-13 * E0
    assert np.max(np.abs(st["TL"] - T0)) > 0.1          # the field did evolve
    q, Q = u.flux(st["I"])
    scale = np.max(np.abs(q))
    assert np.max(np.abs(Q)) <= 1e-12 * scale * np.max(np.linalg.norm(m.nA, axis=1))  # no net flow through the walls


def test_closed_tetrahedral_box_conserves_energy_with_diffuse_and_partial_walls():
    m = M.tet_box(3, 2, 2, 30e-9, 20e-9, 20e-9)
    bands = W.make_bands(3, 1, 17)
    walls = {0: (O.DIFFUSE, None), 1: (O.PARTIAL, 0.3), 2: (O.SPECULAR, None), 3: (O.PARTIAL, 0.8),
             4: (O.DIFFUSE, None), 5: (O.SPECULAR, None)}
    u = O.UMeshProblem(m, O.dirs_for(W.Dirs("polar_azim", n_polar=4, n_azim=8)), bands, walls)
    st = u.init_state(W.random_temperatures(m.ncells, 18, 290.0, 310.0))

    def total(I):
        return sum(m.volume[P] * u.cell_energy(I[P])[0] for P in range(m.ncells))
    E0 = total(st["I"])
    T0 = st["TL"].copy()
    u.run(st, 1e-13, 30, 1, O.EXPLICIT)
    assert abs(total(st["I"]) - E0) <= 1e-13 * E0
    assert np.max(np.abs(st["TL"] - T0)) > 0.1          # the field did evolve
    q, Q = u.flux(st["I"])
    assert np.max(np.abs(Q)) <= 1e-12 * np.max(np.abs(q)) * np.max(np.linalg.norm(m.nA, axis=1))


def test_partial_walls_at_p_one_and_zero_are_the_mirror_and_the_diffuse_wall_bit_for_bit():
    m = M.tri_grid(5, 4, 50e-9, 40e-9, jitter=0.3, seed=8)
    bands, dirs = W.make_bands(4, 1, 14), O.dirs_inplane(12)
    T0 = W.random_temperatures(m.ncells, 15, 296.0, 306.0)
    for p, kind in ((1.0, O.SPECULAR), (0.0, O.DIFFUSE)):
        res = []
        for wall in ((O.PARTIAL, p), (kind, None)):
            u = O.UMeshProblem(m, dirs, bands, {0: (O.ISOTHERMAL, 308.0), 1: (O.ISOTHERMAL, 300.0), 2: wall, 3: wall})
            st = u.init_state(T0)
            u.run(st, 1e-12, 3, 4)
            res.append(st["I"])
        assert np.array_equal(res[0], res[1]), p


def test_per_face_specularity_equal_on_every_face_is_the_uniform_wall():
    m = M.tri_grid(5, 4, 50e-9, 40e-9, jitter=0.3, seed=9)
    bands, dirs = W.make_bands(4, 1, 15), O.dirs_inplane(12)
    T0 = W.random_temperatures(m.ncells, 16, 296.0, 306.0)
    p_faces = np.full(m.nfaces, 0.35)
    res = []
    for p in (0.35, p_faces):
        u = O.UMeshProblem(m, dirs, bands, {0: (O.ISOTHERMAL, 308.0), 1: (O.ISOTHERMAL, 300.0),
                                            2: (O.PARTIAL, p), 3: (O.SPECULAR, None)})
        st = u.init_state(T0)
        u.run(st, 1e-12, 2, 3)
        res.append(st["I"])
    assert np.array_equal(res[0], res[1])


def test_rotating_the_mesh_by_a_quarter_turn_relabels_the_solution():
    """The in-plane set with n % 4 == 0 is invariant under a 90-degree turn, so
    turning the mesh (and its walls) leaves every cell's temperature unchanged."""
    nx, ny, L = 5, 4, 10e-9
    pts, el, _ = _elements_of_tri_grid(nx, ny, nx * L, ny * L)
    rng = np.random.default_rng(11)
    inner = (pts[:, 0] > 0) & (pts[:, 0] < nx * L) & (pts[:, 1] > 0) & (pts[:, 1] < ny * L)
    pts[inner, :2] += rng.uniform(-0.2, 0.2, (inner.sum(), 2)) * L
    vid = lambda i, j: j * (nx + 1) + i
    bnd = {}
    for j in range(ny):
        bnd[frozenset((vid(0, j), vid(0, j + 1)))] = 0
        bnd[frozenset((vid(nx, j), vid(nx, j + 1)))] = 1
    for i in range(nx):
        bnd[frozenset((vid(i, 0), vid(i + 1, 0)))] = 2
        bnd[frozenset((vid(i, ny), vid(i + 1, ny)))] = 3
    a = M.from_elements(pts, el, bnd)
    rot = pts.copy()
    rot[:, 0], rot[:, 1] = -pts[:, 1], pts[:, 0]
    b = M.from_elements(rot, el, bnd)  # the same tags now sit on the turned sides
    bands = W.make_bands(5, 2, 12)
    dirs = O.dirs_inplane(16)
    bc = {0: (O.ISOTHERMAL, 312.0), 1: (O.ISOTHERMAL, 300.0), 2: (O.SPECULAR, None), 3: (O.DIFFUSE, None)}
    # the same walls by tag: the mirror on tag 2 now reflects across x instead of y
    T0 = W.random_temperatures(a.ncells, 13, 299.0, 303.0)
    ua, ub = O.UMeshProblem(a, dirs, bands, bc), O.UMeshProblem(b, dirs, bands, bc)
    sa, sb = ua.init_state(T0), ub.init_state(T0)
    ua.run(sa, 1e-12, 3, 6)
    ub.run(sb, 1e-12, 3, 6)
    assert np.max(np.abs(sa["TL"] - sb["TL"]) / sa["TL"]) < 1e-13
    assert np.max(np.abs(sa["Tp"] - sb["Tp"]) / sa["Tp"]) < 1e-13


def test_the_c_abi_rejects_bad_mesh_descriptions():
    """Argument checks of bte_umesh_create run before any CUDA call."""
    import ctypes as C
    from paper_2305_19400_gb300 import build as B, bte
    B.build()
    L = bte.lib()
    m = M.tri_grid(2, 2, 20e-9, 20e-9)

    def create(**change):
        arr = {"volume": m.volume.copy(), "owner": m.owner.copy(), "neighbor": m.neighbor.copy(),
               "nA": m.nA.copy(), "tag": m.tag.copy()}
        dim = change.pop("dim", 2)
        for k, v in change.items():
            v(arr[k])
        d = bte.bte_umesh_desc()
        d.dim, d.ncells, d.nfaces = dim, m.ncells, m.nfaces
        keep = [np.ascontiguousarray(arr[k], dtype=t) for k, t in
                (("volume", np.float64), ("owner", np.int64), ("neighbor", np.int64), ("nA", np.float64), ("tag", np.int32))]
        d.volume = keep[0].ctypes.data_as(C.POINTER(C.c_double))
        d.owner = keep[1].ctypes.data_as(C.POINTER(C.c_longlong))
        d.neighbor = keep[2].ctypes.data_as(C.POINTER(C.c_longlong))
        d.nA = keep[3].ctypes.data_as(C.POINTER(C.c_double))
        d.tag = keep[4].ctypes.data_as(C.POINTER(C.c_int))
        o = bte.bte_default_opts()
        h = C.c_void_p()
        return L.bte_umesh_create(C.byref(d), C.byref(o), C.byref(h)), h

    def setv(idx, val):
        def f(a):
            a[idx] = val
        return f
    for change in ({"dim": 4}, {"volume": setv(0, -1.0)}, {"owner": setv(0, m.ncells)},
                   {"neighbor": setv(int(np.nonzero(m.neighbor >= 0)[0][0]), int(m.owner[np.nonzero(m.neighbor >= 0)[0][0]]))},
                   {"nA": setv((0, 2), 1e-9)}, {"tag": setv(int(m.boundary_faces()[0]), -3)}):
        rc, h = create(**change)
        assert rc == -1 and not h.value, change
    o = bte.bte_default_opts()
    o.precision = bte.BTE_FP32
    d = bte.bte_umesh_desc()
    h = C.c_void_p()
    assert L.bte_umesh_create(None, C.byref(o), C.byref(h)) == -1
    assert b"NULL" in L.bte_umesh_last_error(None)
