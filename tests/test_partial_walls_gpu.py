"""Partially specular walls (bte_set_specularity) through the C ABI against the
FP64 oracle.

A side with specularity p gives every incoming direction p x the wall cell's
mirrored value + (1 - p) x its diffuse value.  Checks: FP64 parity (rel 1e-12
on T, 1e-11 on I) with point-Jacobi and sweep-ordered inner iterations, the
p = 1 and p = 0 limits against mirror and diffuse walls, FP32 in 3-D within
1e-4 K, BF16 within its reported error, zero net flux through the walls, and
graph replay, including a specularity changed after a capture.  The same on
unstructured meshes (bte_umesh_set_bc with BTE_BC_PARTIAL): FP64 parity with
implicit and explicit steps and a specularity that varies along a wall, the
limits bit for bit in FP64 and FP32, FP32 / BF16 storage, and a specularity
changed between steps.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O
from paper_2305_19400_gb300 import bte, workloads as W

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2305_19400_gb300 import build as B
    B.build()
    O.build()


def channel(p_spec, nx=19, ny=13):
    wl = W.cfg2(nx, ny)
    g = wl.geoms[0]
    g.bc[2] = (W.BC_PARTIAL, p_spec)
    g.bc[3] = (W.BC_PARTIAL, p_spec)
    return wl


def oracle_of(wl, nsteps, ninner, scheme=O.IMPLICIT):
    g = wl.geoms[0]
    p = O.Problem(g, O.dirs_for(wl.dirs), wl.bands)
    st = p.init_state(g.T_init)
    p.run(st, wl.dt, nsteps, ninner, scheme)
    return p, st


@pytest.mark.parametrize("scheme", [bte.BTE_IMPLICIT_JACOBI, bte.BTE_IMPLICIT_GS])
def test_fp64_partially_specular_channel_matches_oracle(scheme):
    wl = channel(0.35)
    s = bte.Solver(wl)
    rc, st = s.step(nsteps=3, ninner=8, scheme=scheme)
    assert rc >= 0 and st["nonfinite"] == 0
    per_iter = (2 if scheme == bte.BTE_IMPLICIT_JACOBI else 3) + 2          # + the two ghost-row refreshes
    assert st["launches"] == 3 * 8 * per_iter
    p, ost = oracle_of(wl, 3, 8, O.GAUSS_SEIDEL if scheme == bte.BTE_IMPLICIT_GS else O.IMPLICIT)
    for which, key in ((bte.BTE_T_LATTICE, "TL"), (bte.BTE_T_PSEUDO, "Tp")):
        assert np.max(np.abs(s.T(0, which) - ost[key]) / ost[key]) <= 1e-12, key
    assert np.max(np.abs(s.intensity(0) - ost["I"]) / np.abs(ost["I"])) <= 1e-11
    q, qw = s.flux(0)
    q_ref, qw_ref = p.flux(ost["I"])
    scale = np.max(np.abs(q_ref))
    assert np.max(np.abs(q - q_ref)) <= 1e-10 * scale
    assert np.max(np.abs(qw - qw_ref)) <= 1e-10 * scale
    assert np.all(np.abs(qw[2:]) <= 1e-10 * scale)         # no net flux through the partial walls
    s.close()


def test_the_limits_are_the_mirror_and_the_diffuse_wall():
    for p_spec, kind in ((1.0, W.BC_SPECULAR), (0.0, W.BC_DIFFUSE)):
        a = bte.Solver(channel(p_spec, 11, 7))
        wl = W.cfg2(11, 7)
        wl.geoms[0].bc[2] = (kind, None)
        wl.geoms[0].bc[3] = (kind, None)
        b = bte.Solver(wl)
        a.step(nsteps=2, ninner=5)
        b.step(nsteps=2, ninner=5)
        Ia, Ib = a.intensity(0), b.intensity(0)
        assert np.max(np.abs(Ia - Ib) / Ib) <= 1e-13, p_spec
        a.close()
        b.close()


@pytest.mark.parametrize("precision,tol", [(bte.BTE_FP32, 1e-4), (bte.BTE_BF16, 1e-3)])
def test_reduced_precision_3d_partial_walls(precision, tol):
    g = W.Geometry(3, 6, 5, 4, 10e-9, 10e-9, 10e-9)
    W.uniform_walls(g, [W.BC_ISOTHERMAL, W.BC_ISOTHERMAL, W.BC_SPECULAR, W.BC_SPECULAR, W.BC_PARTIAL, W.BC_PARTIAL],
                    [306.0, 300.0, 0, 0, 0.6, 0.6])
    wl = W.Workload("3d partial", [g], W.Dirs("polar_azim", n_polar=4, n_azim=8), W.make_bands(8, 3, 52), 1e-12, 3, 6)
    s = bte.Solver(wl, precision=precision)
    s.step(nsteps=3, ninner=6)
    _, ost = oracle_of(wl, 3, 6)
    assert np.max(np.abs(s.T(0, bte.BTE_T_LATTICE) - ost["TL"])) <= tol
    assert np.max(np.abs(s.T(0, bte.BTE_T_PSEUDO) - ost["Tp"])) <= tol
    s.close()


def test_graph_replay_and_a_specularity_changed_after_capture():
    eager = bte.Solver(channel(0.5, 9, 7))
    graph = bte.Solver(channel(0.5, 9, 7), use_graph=True)
    for s in (eager, graph):
        s.step(nsteps=2, ninner=4)
    assert np.array_equal(eager.intensity(0), graph.intensity(0))
    for s in (eager, graph):  # the captured step carries p: a new p must not replay the old graph
        for side in (2, 3):
            assert bte.lib().bte_set_specularity(s.h, 0, side, 0.2) == 0
        s.step(nsteps=2, ninner=4)
    assert np.array_equal(eager.intensity(0), graph.intensity(0))
    wl = channel(0.5, 9, 7)   # the oracle with p = 0.5 for two steps, then 0.2
    g = wl.geoms[0]
    p = O.Problem(g, O.dirs_for(wl.dirs), wl.bands)
    st = p.init_state(g.T_init)
    p.run(st, wl.dt, 2, 4)
    g.bc[2] = (W.BC_PARTIAL, 0.2)
    g.bc[3] = (W.BC_PARTIAL, 0.2)
    p2 = O.Problem(g, O.dirs_for(wl.dirs), wl.bands)
    p2.run(st, wl.dt, 2, 4)
    assert np.max(np.abs(eager.T(0, bte.BTE_T_LATTICE) - st["TL"]) / st["TL"]) <= 1e-12
    assert bte.lib().bte_set_specularity(eager.h, 0, 2, 1.5) == -1
    eager.close()
    graph.close()


# ----------------------------------------------------------- unstructured meshes
from paper_2305_19400_gb300 import mesh as M  # noqa: E402


def umesh_case(p_lo=0.3, p_hi=None):
    """Jittered triangles, 400 directions x 55 bands, a hot and a cold wall and
    two partially specular walls (tags 2 and 3; tag 3's specularity varies
    along the wall when p_hi is given)."""
    m = M.tri_grid(13, 9, 130e-9, 90e-9, jitter=0.3, seed=23)
    p3 = 0.7
    if p_hi is not None:
        p3 = np.zeros(m.nfaces)
        f = m.boundary_faces(3)
        x = m.face_center[f, 0]
        p3[f] = p_lo + (p_hi - p_lo) * (x - x.min()) / np.ptp(x)
    bc = {0: (bte.BTE_BC_ISOTHERMAL, 308.0), 1: (bte.BTE_BC_ISOTHERMAL, 300.0),
          2: (bte.BTE_BC_PARTIAL, p_lo), 3: (bte.BTE_BC_PARTIAL, p3)}
    return m, W.Dirs("polar_azim", n_polar=20, n_azim=20), W.make_bands(40, 15, 19407), bc


def umesh_oracle(m, dirs, bands, bc, dt, nsteps, ninner, scheme):
    u = O.UMeshProblem(m, O.dirs_for(dirs), bands, bc)
    ost = u.init_state(m.T_init)
    u.run(ost, dt, nsteps, ninner, O.EXPLICIT if scheme == bte.BTE_EXPLICIT else O.IMPLICIT)
    return u, ost


@pytest.mark.parametrize("scheme,dt,nsteps,ninner", [(bte.BTE_IMPLICIT_JACOBI, 1e-12, 3, 5),
                                                     (bte.BTE_EXPLICIT, 2e-13, 12, 1)])
def test_fp64_unstructured_partial_walls_match_oracle(scheme, dt, nsteps, ninner):
    m, dirs, bands, bc = umesh_case(0.3, 0.9)
    s = bte.UMeshSolver(m, dirs, bands, bc)
    rc, st = s.step(dt, nsteps, ninner, scheme)
    assert rc >= 0 and st["nonfinite"] == 0
    u, ost = umesh_oracle(m, dirs, bands, bc, dt, nsteps, ninner, scheme)
    for which, key in ((bte.BTE_T_LATTICE, "TL"), (bte.BTE_T_PSEUDO, "Tp")):
        assert np.max(np.abs(s.T(which) - ost[key]) / ost[key]) <= 1e-12, key
    assert np.max(np.abs(s.intensity() - ost["I"]) / np.abs(ost["I"])) <= 1e-11
    q, Q = s.flux()
    q_ref, Q_ref = u.flux(ost["I"])
    assert np.max(np.abs(q - q_ref)) <= 1e-10 * np.max(np.abs(q_ref))
    assert np.max(np.abs(Q - Q_ref)) <= 1e-10 * np.max(np.abs(Q_ref))
    partial = np.concatenate([m.boundary_faces(2), m.boundary_faces(3)])
    assert np.max(np.abs(Q[partial])) <= 1e-10 * np.max(np.abs(Q_ref))   # no net flow through them
    s.close()


@pytest.mark.parametrize("precision", [bte.BTE_FP64, bte.BTE_FP32])
def test_unstructured_limits_are_the_mirror_and_the_diffuse_wall_bit_for_bit(precision):
    m = M.tri_grid(7, 5, 70e-9, 50e-9, jitter=0.3, seed=24)
    dirs, bands = W.Dirs("inplane", n_inplane=16), W.make_bands(6, 2, 65)
    for p_spec, kind in ((1.0, bte.BTE_BC_SPECULAR), (0.0, bte.BTE_BC_DIFFUSE)):
        out = []
        for wall in ((bte.BTE_BC_PARTIAL, p_spec), (kind, None)):
            s = bte.UMeshSolver(m, dirs, bands, {0: (0, 309.0), 1: (0, 300.0), 2: wall, 3: wall}, precision=precision)
            s.step(1e-12, 3, 5)
            out.append(s.intensity())
            s.close()
        assert np.array_equal(out[0], out[1]), p_spec


@pytest.mark.parametrize("precision,tol", [(bte.BTE_FP32, 1e-4), (bte.BTE_BF16, 2e-3)])
def test_reduced_storage_unstructured_partial_walls(precision, tol):
    m, dirs, bands, bc = umesh_case(0.4)
    s = bte.UMeshSolver(m, dirs, bands, bc, precision=precision)
    rc, st = s.step(1e-12, 3, 8)
    assert rc >= 0 and st["nonfinite"] == 0
    u, ost = umesh_oracle(m, dirs, bands, bc, 1e-12, 3, 8, bte.BTE_IMPLICIT_JACOBI)
    assert np.max(np.abs(s.T(bte.BTE_T_LATTICE) - ost["TL"])) <= tol
    assert np.max(np.abs(s.T(bte.BTE_T_PSEUDO) - ost["Tp"])) <= tol
    _, Q = s.flux()
    _, Q_ref = u.flux(ost["I"])
    assert np.max(np.abs(Q - Q_ref)) <= 100 * tol * np.max(np.abs(Q_ref))
    s.close()


def test_unstructured_specularity_changed_between_steps_and_bad_values():
    m, dirs, bands, bc = umesh_case(0.5)
    s = bte.UMeshSolver(m, dirs, bands, bc)
    s.step(1e-12, 2, 4)
    s.set_bc(2, bte.BTE_BC_PARTIAL, 0.1)
    s.step(1e-12, 2, 4)
    u = O.UMeshProblem(m, O.dirs_for(dirs), bands, bc)
    ost = u.init_state(m.T_init)
    u.run(ost, 1e-12, 2, 4)
    bc2 = dict(bc)
    bc2[2] = (bte.BTE_BC_PARTIAL, 0.1)
    O.UMeshProblem(m, O.dirs_for(dirs), bands, bc2).run(ost, 1e-12, 2, 4)
    assert np.max(np.abs(s.T(bte.BTE_T_LATTICE) - ost["TL"]) / ost["TL"]) <= 1e-12
    for bad in (-0.1, 1.5, float("nan")):
        with pytest.raises(bte.BTEError) as e:
            s.set_bc(2, bte.BTE_BC_PARTIAL, bad)
        assert e.value.code == -1
    s.step(1e-12, 1, 4)                                  # the refused calls changed nothing
    O.UMeshProblem(m, O.dirs_for(dirs), bands, bc2).run(ost, 1e-12, 1, 4)
    assert np.max(np.abs(s.T(bte.BTE_T_LATTICE) - ost["TL"]) / ost["TL"]) <= 1e-12
    s.close()
