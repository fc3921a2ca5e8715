"""Diffuse (rough) walls through the C ABI against the FP64 oracle.

A diffuse wall gives every incoming direction of a band the same intensity,
sum_out |S.n| I / sum_in |S.n| of the wall cell's current iterate.  The GPU
refreshes these ghosts before every sweep; checks: FP64 parity (rel 1e-12 on
T, 1e-11 on I) in 2-D and 3-D, FP32 within 1e-4 K, energy conservation in a
diffuse box, zero net flux through diffuse walls, graph replay equal to eager
launches.
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


def channel(nx=17, ny=11):
    """The 400-direction hot-spot channel with rough side walls."""
    wl = W.cfg2(nx, ny)
    g = wl.geoms[0]
    g.bc[2] = (W.BC_DIFFUSE, None)
    g.bc[3] = (W.BC_DIFFUSE, None)
    return wl


def oracle_of(wl, nsteps, ninner, scheme=O.IMPLICIT, dt=None, T_init=None):
    g = wl.geoms[0]
    p = O.Problem(g, O.dirs_for(wl.dirs), wl.bands)
    st = p.init_state(g.T_init if T_init is None else T_init)
    p.run(st, wl.dt if dt is None else dt, nsteps, ninner, scheme)
    return p, st


def test_fp64_channel_with_rough_side_walls_matches_oracle():
    wl = channel()
    s = bte.Solver(wl)
    rc, st = s.step(nsteps=3, ninner=10)
    assert rc >= 0 and st["nonfinite"] == 0
    assert st["launches"] == 3 * 10 * (2 + 2)            # sweep, fix-up and the two diffuse ghost rows
    p, ost = oracle_of(wl, 3, 10)
    for which, key in ((bte.BTE_T_LATTICE, "TL"), (bte.BTE_T_PSEUDO, "Tp")):
        assert np.max(np.abs(s.T(0, which) - ost[key]) / ost[key]) <= 1e-12, key
    I = s.intensity(0)
    assert np.max(np.abs(I - ost["I"]) / np.abs(ost["I"])) <= 1e-11
    q, qw = s.flux(0)
    q_ref, qw_ref = p.flux(ost["I"])
    scale = np.max(np.abs(q_ref))
    assert np.max(np.abs(q - q_ref)) <= 1e-10 * scale
    assert np.max(np.abs(qw - qw_ref)) <= 1e-10 * scale
    assert np.all(np.abs(qw[2:]) <= 1e-10 * scale)        # no net flux through the rough walls
    # the rough walls change the answer (against mirror walls)
    _, mirror = oracle_of(W.cfg2(17, 11), 3, 10)
    assert np.max(np.abs(mirror["TL"] - ost["TL"])) > 1e-6
    s.close()


def test_fp32_channel_with_rough_side_walls_within_tolerance():
    wl = channel()
    s = bte.Solver(wl, precision=bte.BTE_FP32)
    s.step(nsteps=3, ninner=10)
    _, ost = oracle_of(wl, 3, 10)
    assert np.max(np.abs(s.T(0, bte.BTE_T_LATTICE) - ost["TL"])) <= 1e-4
    assert np.max(np.abs(s.T(0, bte.BTE_T_PSEUDO) - ost["Tp"])) <= 1e-4
    s.close()


def test_fp64_3d_rough_z_walls_match_oracle():
    g = W.Geometry(3, 5, 4, 3, 10e-9, 10e-9, 10e-9)
    W.uniform_walls(g, [W.BC_ISOTHERMAL, W.BC_ISOTHERMAL, W.BC_SPECULAR, W.BC_SPECULAR, W.BC_DIFFUSE, W.BC_DIFFUSE],
                    [306.0, 300.0, 0, 0, 0, 0])
    wl = W.Workload("3d rough", [g], W.Dirs("polar_azim", n_polar=4, n_azim=8), W.make_bands(8, 3, 52), 1e-12, 3, 6)
    s = bte.Solver(wl)
    s.step(nsteps=3, ninner=6)
    _, ost = oracle_of(wl, 3, 6)
    assert np.max(np.abs(s.T(0, bte.BTE_T_LATTICE) - ost["TL"]) / ost["TL"]) <= 1e-12
    assert np.max(np.abs(s.intensity(0) - ost["I"]) / np.abs(ost["I"])) <= 1e-11
    g2 = W.Geometry(3, 5, 4, 3, 10e-9, 10e-9, 10e-9)      # the same with mirror z walls differs
    W.uniform_walls(g2, [W.BC_ISOTHERMAL, W.BC_ISOTHERMAL] + [W.BC_SPECULAR] * 4, [306.0, 300.0, 0, 0, 0, 0])
    _, mirror = oracle_of(W.Workload("3d mirror", [g2], wl.dirs, wl.bands, 1e-12, 3, 6), 3, 6)
    assert np.max(np.abs(mirror["TL"] - ost["TL"])) > 1e-4
    s.close()


def test_diffuse_box_conserves_energy_on_gpu():
    g = W.Geometry(2, 6, 5, 1, 10e-9, 10e-9, 10e-9)
    W.uniform_walls(g, [W.BC_DIFFUSE] * 4, [0.0] * 4)
    wl = W.Workload("rough box", [g], W.Dirs("polar_azim", n_polar=4, n_azim=8), W.make_bands(6, 2, 53), 2e-13, 80, 1)
    T0 = W.random_temperatures(30, 13, 285.0, 320.0)
    s = bte.Solver(wl, T_init=[T0])
    p = O.Problem(g, O.dirs_for(wl.dirs), wl.bands)
    E0 = sum(p.cell_energy(r)[0] for r in s.intensity(0))
    s.step(scheme=bte.BTE_EXPLICIT)
    E1 = sum(p.cell_energy(r)[0] for r in s.intensity(0))
    assert abs(E1 - E0) <= 1e-13 * E0
    s.close()


def test_graph_replay_includes_the_ghost_refresh():
    wl = channel(9, 7)
    eager = bte.Solver(wl)
    graph = bte.Solver(wl, use_graph=True)
    for nsteps, ninner in ((1, 5), (2, 5)):
        eager.step(nsteps=nsteps, ninner=ninner)
        graph.step(nsteps=nsteps, ninner=ninner)
    assert np.array_equal(eager.intensity(0), graph.intensity(0))
    eager.close(); graph.close()
