"""Sweep-ordered (Gauss-Seidel) inner iterations through the C ABI against the
FP64 oracle's sweep-ordered mode.

Bar (FP64): temperatures within rel 1e-12, intensities within rel 1e-11, on a
ragged 2-D grid with 400 directions x 55 band-pols, a 3-D grid with
isothermal, mirror and diffuse walls, several geometries in one handle, and
temperature-dependent relaxation.  The pass's results do not depend on the CTA
layout or tile size (each (d, b) is the same triangular solve), so graph
replay and autotuned layouts must agree bitwise.  At the full 128x128 x 400 x
55 size, sampled outputs of one pass are checked against the sweep-ordered
update written out by the oracle, with the GPU's own pass as the upwind field.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O
from paper_2305_19400_gb300 import bte, workloads as W

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

GS = bte.BTE_IMPLICIT_GS


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2305_19400_gb300 import build as B
    B.build()
    O.build()


def oracle_run(wl, nsteps, ninner, geom_index=0, T_init=None, beta_exp=0.0, scheme=O.GAUSS_SEIDEL):
    g = wl.geoms[geom_index]
    p = O.Problem(g, O.dirs_for(wl.dirs), wl.bands, beta_exp=beta_exp, beta_Tref=300.0)
    st = p.init_state(g.T_init if T_init is None else T_init)
    p.run(st, wl.dt, nsteps, ninner, scheme)
    return p, st


def assert_matches(s, ost, gi=0):
    for which, key in ((bte.BTE_T_LATTICE, "TL"), (bte.BTE_T_PSEUDO, "Tp")):
        T = s.T(gi, which)
        assert np.max(np.abs(T - ost[key]) / ost[key]) <= 1e-12, key
    I = s.intensity(gi)
    assert np.max(np.abs(I - ost["I"]) / np.abs(ost["I"])) <= 1e-11


def test_ragged_2d_grid_400_directions_matches_oracle():
    wl = W.cfg2(19, 13)
    s = bte.Solver(wl)
    rc, st = s.step(nsteps=3, ninner=6, scheme=GS)
    assert rc >= 0 and st["nonfinite"] == 0
    assert st["launches"] == 3 * 6 * 3                     # pass, per-cell step, fix-up
    p, ost = oracle_run(wl, 3, 6)
    assert_matches(s, ost)
    q, qw = s.flux(0)
    q_ref, qw_ref = p.flux(ost["I"])
    scale = np.max(np.abs(q_ref))
    assert np.max(np.abs(q - q_ref)) <= 1e-10 * scale
    # a different iteration from Jacobi's at a finite inner count
    _, jac = oracle_run(wl, 3, 6, scheme=O.IMPLICIT)
    assert np.max(np.abs(jac["TL"] - ost["TL"])) > 1e-6
    s.close()


def test_3d_isothermal_mirror_and_diffuse_walls_match_oracle():
    g = W.Geometry(3, 5, 4, 3, 10e-9, 8e-9, 12e-9)
    g.bc = [(W.BC_ISOTHERMAL, np.full(12, 300.0)), (W.BC_ISOTHERMAL, W.random_temperatures(12, 5, 300.0, 310.0)),
            (W.BC_SPECULAR, None), (W.BC_DIFFUSE, None),
            (W.BC_ISOTHERMAL, np.full(20, 302.0)), (W.BC_SPECULAR, None)]
    wl = W.Workload("3d", [g], W.Dirs("polar_azim", n_polar=4, n_azim=8), W.make_bands(40, 15, 19403), 1e-12, 3, 6)
    T0 = W.random_temperatures(60, 6, 298.0, 303.0)
    s = bte.Solver(wl, T_init=[T0])
    rc, st = s.step(nsteps=3, ninner=6, scheme=GS)
    assert st["launches"] == 3 * 6 * (3 + 1)               # and the diffuse ghost row
    _, ost = oracle_run(wl, 3, 6, T_init=T0)
    assert_matches(s, ost)
    s.close()


def test_3d_grid_larger_than_one_column_tile():
    """17 x 11 x 6 cells: several 8x8 column tiles with ragged last ones."""
    g = W.Geometry(3, 17, 11, 6, 10e-9, 10e-9, 10e-9)
    W.uniform_walls(g, [W.BC_ISOTHERMAL, W.BC_ISOTHERMAL] + [W.BC_SPECULAR] * 4, [306.0, 300.0, 0, 0, 0, 0])
    wl = W.Workload("3d tiles", [g], W.Dirs("polar_azim", n_polar=4, n_azim=8), W.make_bands(8, 3, 52), 1e-12, 2, 4)
    s = bte.Solver(wl)
    s.step(nsteps=2, ninner=4, scheme=GS)
    _, ost = oracle_run(wl, 2, 4)
    assert_matches(s, ost)
    s.close()


def test_several_geometries_in_one_handle_match_oracle_one_by_one():
    geoms = []
    for (nx, ny, th) in ((7, 5, 312.0), (1, 1, 305.0), (13, 3, 301.5), (2, 9, 318.0)):
        g = W.Geometry(2, nx, ny, 1, 10e-9, 10e-9, 10e-9)
        W.uniform_walls(g, [W.BC_ISOTHERMAL, W.BC_ISOTHERMAL, W.BC_SPECULAR, W.BC_SPECULAR], [th, 300.0, 0, 0])
        geoms.append(g)
    geoms[2].dx = 7e-9  # a second cell-size class
    wl = W.Workload("batch", geoms, W.Dirs("inplane", n_inplane=16), W.make_bands(40, 15, 19405), 1e-12, 4, 5)
    s = bte.Solver(wl)
    s.step(nsteps=4, ninner=5, scheme=GS)
    for gi in range(len(geoms)):
        _, ost = oracle_run(wl, 4, 5, geom_index=gi)
        assert_matches(s, ost, gi)
    s.close()


def test_temperature_dependent_relaxation_matches_oracle():
    wl = W.cfg2(13, 9)
    g = wl.geoms[0]
    T0 = W.random_temperatures(g.ncells, 17, 320.0, 340.0)
    s = bte.Solver(wl, beta_exp=1.0, T_ref=300.0, T_init=[T0])
    rc, st = s.step(nsteps=4, ninner=8, scheme=GS)
    assert st["launches"] == 4 * 8 * 4                     # and the per-cell rate factor
    _, ost = oracle_run(wl, 4, 8, T_init=T0, beta_exp=1.0)
    assert_matches(s, ost)
    s.close()


def test_graph_replay_and_autotuned_layouts_agree_bitwise():
    wl = W.cfg2(21, 10)
    eager = bte.Solver(wl)
    graph = bte.Solver(wl, use_graph=True)
    tuned = bte.Solver(wl, use_graph=True, autotune=True)
    for s in (eager, graph, tuned):
        s.step(nsteps=2, ninner=4, scheme=GS)
        s.step(nsteps=1, ninner=4, scheme=GS)
    ref = eager.intensity(0)
    assert np.array_equal(graph.intensity(0), ref)
    assert np.array_equal(tuned.intensity(0), ref)
    report = bte.bte_autotune(tuned.h, wl.dt, GS)
    assert report.startswith("directions_per_cta") and "chosen" in report
    for s in (eager, graph, tuned):
        s.close()


def test_fewer_inner_iterations_than_jacobi_for_the_same_error():
    """Same converged step; after 4 inner iterations the sweep-ordered T_L is
    closer to it than Jacobi's (on the GPU, both schemes)."""
    wl = W.cfg2(19, 13)
    ref = bte.Solver(wl)
    ref.step(nsteps=1, ninner=40, scheme=GS)
    T_ref = ref.T(0, bte.BTE_T_LATTICE)
    errs = {}
    for scheme in (GS, bte.BTE_IMPLICIT_JACOBI):
        s = bte.Solver(wl)
        s.step(nsteps=1, ninner=4, scheme=scheme)
        errs[scheme] = np.max(np.abs(s.T(0, bte.BTE_T_LATTICE) - T_ref))
        s.close()
    assert errs[GS] < 0.7 * errs[bte.BTE_IMPLICIT_JACOBI], errs
    ref.close()


@pytest.mark.parametrize("precision,tol", [(bte.BTE_FP32, 1e-4), (bte.BTE_BF16, 2e-3)])
def test_reduced_storage_sweep_ordered_pass(precision, tol):
    """FP32 (BF16) deviation storage with sweep-ordered iterations against the
    FP64 oracle's sweep-ordered mode: 2-D with diffuse and partial walls,
    3-D with mirror walls, and tau(T).  BF16 only near T_ref: cells 20-40 K
    away carry deviations whose 8-bit rounding alone exceeds its bound."""
    wl = W.cfg2(19, 13)
    wl.geoms[0].bc[2] = (W.BC_DIFFUSE, None)
    wl.geoms[0].bc[3] = (W.BC_PARTIAL, 0.4)
    s = bte.Solver(wl, precision=precision)
    s.step(nsteps=3, ninner=6, scheme=GS)
    _, ost = oracle_run(wl, 3, 6)
    assert np.max(np.abs(s.T(0, bte.BTE_T_LATTICE) - ost["TL"])) <= tol
    assert np.max(np.abs(s.T(0, bte.BTE_T_PSEUDO) - ost["Tp"])) <= tol
    s.close()
    if precision == bte.BTE_BF16:
        return
    g = W.Geometry(3, 9, 7, 5, 10e-9, 10e-9, 10e-9)
    W.uniform_walls(g, [W.BC_ISOTHERMAL, W.BC_ISOTHERMAL] + [W.BC_SPECULAR] * 4, [306.0, 300.0, 0, 0, 0, 0])
    wl3 = W.Workload("3d", [g], W.Dirs("polar_azim", n_polar=4, n_azim=8), W.make_bands(8, 3, 52), 1e-12, 2, 4)
    s = bte.Solver(wl3, precision=precision)
    s.step(nsteps=2, ninner=4, scheme=GS)
    _, ost = oracle_run(wl3, 2, 4)
    assert np.max(np.abs(s.T(0, bte.BTE_T_LATTICE) - ost["TL"])) <= tol
    s.close()
    wlt = W.cfg2(13, 9)
    T0 = W.random_temperatures(wlt.geoms[0].ncells, 17, 320.0, 340.0)
    s = bte.Solver(wlt, precision=precision, beta_exp=1.0, T_ref=300.0, T_init=[T0])
    s.step(nsteps=3, ninner=6, scheme=GS)
    _, ost = oracle_run(wlt, 3, 6, T_init=T0, beta_exp=1.0)
    assert np.max(np.abs(s.T(0, bte.BTE_T_LATTICE) - ost["TL"])) <= tol
    s.close()


def test_full_size_pass_sampled_against_oracle():
    """128x128 x 400 x 55 (the benchmark's workload), graph replay and the
    autotuned layout: one pass from the step's start, checked at sampled
    (P, d, b) (every corner and edge-middle cell, random interior cells)
    against the sweep-ordered update with the GPU's own pass as the field of
    upwind values; temperatures of the sampled cells from their rows."""
    wl = W.cfg2()
    g = wl.geoms[0]
    s = bte.Solver(wl, use_graph=True, autotune=True)
    s.step(nsteps=1, ninner=3, scheme=GS)
    I_n = s.intensity(0)
    Tp_n = s.T(0, bte.BTE_T_PSEUDO)
    s.step(nsteps=1, ninner=1, scheme=GS)
    I_1 = s.intensity(0)
    Tp_1 = s.T(0, bte.BTE_T_PSEUDO)
    TL_1 = s.T(0, bte.BTE_T_LATTICE)
    p = O.Problem(g, O.dirs_for(wl.dirs), wl.bands)
    rng = np.random.default_rng(3)
    nc, nd, nb = I_n.shape
    cells = set(rng.integers(0, nc, 40).tolist())
    cells |= {0, g.nx - 1, nc - g.nx, nc - 1, g.nx // 2, nc - g.nx // 2, (g.ny // 2) * g.nx,
              (g.ny // 2) * g.nx + g.nx - 1}
    I0 = np.zeros((nc, nb))
    for P in cells:
        I0[P] = O.I0(wl.bands, Tp_n[P])[0]
    I0w = p.wall_I0()
    worst = 0.0
    for P in sorted(cells):
        for d in rng.integers(0, nd, 12):
            for b in rng.integers(0, nb, 4):
                ref = p.gs_update_one(wl.dt, I_n, I_n, I_1, I0, I0w, P, d, b)
                worst = max(worst, abs(I_1[P, d, b] - ref) / abs(ref))
        Tp_ref, TL_ref = p.cell_temperatures(I_1[P], Tp_n[P], Tp_n[P])
        assert abs(Tp_1[P] - Tp_ref) <= 1e-12 * Tp_ref
        assert abs(TL_1[P] - TL_ref) <= 1e-12 * TL_ref
    assert worst <= 1e-12, worst
    s.close()


@pytest.mark.parametrize("dims,nbands,dirs", [((2, 1, 1, 1), 4, W.Dirs("inplane", n_inplane=8)),
                                              ((2, 9, 1, 1), 1, W.Dirs("inplane", n_inplane=12)),
                                              ((3, 1, 1, 5), 3, W.Dirs("polar_azim", n_polar=4, n_azim=8)),
                                              ((2, 3, 2, 1), 3, W.Dirs("polar_azim", n_polar=32, n_azim=64))])
def test_degenerate_grids_one_band_and_the_largest_direction_set(dims, nbands, dirs):
    dim, nx, ny, nz = dims
    g = W.Geometry(dim, nx, ny, nz, 10e-9, 10e-9, 10e-9)
    kinds = [W.BC_ISOTHERMAL, W.BC_ISOTHERMAL] + [W.BC_SPECULAR] * (2 * dim - 2)
    W.uniform_walls(g, kinds, [305.0, 300.0] + [0.0] * (2 * dim - 2))
    bands = W.make_bands(nbands, 0, 61) if nbands > 1 else W.make_bands(1, 0, 61)
    wl = W.Workload("edge", [g], dirs, bands, 1e-12, 2, 3)
    s = bte.Solver(wl)
    s.step(nsteps=2, ninner=3, scheme=GS)
    _, ost = oracle_run(wl, 2, 3)
    assert_matches(s, ost)
    s.close()
