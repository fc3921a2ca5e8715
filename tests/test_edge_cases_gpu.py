"""Edge cases of the hot path against the FP64 oracle (FP64 mode: rel 1e-12 on
T, 1e-11 on I; FP32: max|dT| <= 1e-4 K): degenerate grids (single cells and
one-cell-wide strips, 2-D and 3-D), one band and the maximum band count, the
largest direction set, every beta_b = 0 (the T_p equation is empty), zero time
steps, and the direction limit."""
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


def compare(wl, nsteps, ninner, precision=bte.BTE_FP64, scheme=bte.BTE_IMPLICIT_JACOBI, T_init=None):
    s = bte.Solver(wl, precision=precision, T_init=T_init)
    rc, st = s.step(nsteps=nsteps, ninner=ninner, scheme=scheme)
    assert rc >= 0 and st["nonfinite"] == 0
    g = wl.geoms[0]
    p = O.Problem(g, O.dirs_for(wl.dirs), wl.bands)
    ost = p.init_state(g.T_init if T_init is None else T_init[0])
    p.run(ost, wl.dt, nsteps, ninner, O.EXPLICIT if scheme == bte.BTE_EXPLICIT else O.IMPLICIT)
    TL, Tp = s.T(0, bte.BTE_T_LATTICE), s.T(0, bte.BTE_T_PSEUDO)
    if precision == bte.BTE_FP64:
        assert np.max(np.abs(TL - ost["TL"]) / ost["TL"]) <= 1e-12
        assert np.max(np.abs(Tp - ost["Tp"]) / ost["Tp"]) <= 1e-12
        I = s.intensity(0)
        assert np.max(np.abs(I - ost["I"]) / np.maximum(np.abs(ost["I"]), 1e-300)) <= 1e-11
    else:
        assert np.max(np.abs(TL - ost["TL"])) <= 1e-4
        assert np.max(np.abs(Tp - ost["Tp"])) <= 1e-4
    s.close()
    return ost


def hot_cold(g):
    kinds = [W.BC_ISOTHERMAL, W.BC_ISOTHERMAL] + [W.BC_SPECULAR] * (2 * g.dim - 2)
    W.uniform_walls(g, kinds, [305.0, 300.0] + [0.0] * (2 * g.dim - 2))
    return g


@pytest.mark.parametrize("dims", [(2, 1, 1, 1), (2, 1, 9, 1), (2, 9, 1, 1), (3, 1, 1, 1), (3, 1, 3, 2), (3, 2, 1, 3)])
def test_degenerate_grids(dims):
    dim, nx, ny, nz = dims
    g = hot_cold(W.Geometry(dim, nx, ny, nz, 10e-9, 10e-9, 10e-9))
    dirs = W.Dirs("inplane", n_inplane=8) if dim == 2 else W.Dirs("polar_azim", n_polar=4, n_azim=8)
    wl = W.Workload("degenerate", [g], dirs, W.make_bands(6, 2, 41), 1e-12, 4, 5)
    ost = compare(wl, 4, 5)
    assert np.max(ost["TL"]) > 300.0          # the hot wall reached the cells


def test_single_band():
    g = hot_cold(W.Geometry(2, 6, 5, 1, 10e-9, 10e-9, 10e-9))
    wl = W.Workload("one band", [g], W.Dirs("inplane", n_inplane=12), W.make_bands(1, 0, 42), 1e-12, 5, 4)
    assert wl.bands.nb == 1
    compare(wl, 5, 4)


@pytest.mark.parametrize("precision", [bte.BTE_FP64, bte.BTE_FP32])
def test_maximum_band_count(precision):
    g = hot_cold(W.Geometry(2, 5, 3, 1, 10e-9, 10e-9, 10e-9))
    wl = W.Workload("256 bands", [g], W.Dirs("inplane", n_inplane=8), W.make_bands(200, 56, 43), 1e-12, 3, 3)
    assert wl.bands.nb == 256
    compare(wl, 3, 3, precision)


def test_largest_direction_set():
    g = hot_cold(W.Geometry(2, 3, 2, 1, 10e-9, 10e-9, 10e-9))
    wl = W.Workload("2048 directions", [g], W.Dirs("polar_azim", n_polar=32, n_azim=64), W.make_bands(3, 1, 44),
                    1e-12, 2, 2)
    assert wl.dirs.nd == 2048
    compare(wl, 2, 2)
    with pytest.raises(bte.BTEError) as e:        # one ring more is refused at initialisation
        o = bte.bte_default_opts()
        o.dir_kind, o.n_polar, o.n_azim = bte.BTE_DIRS_POLAR_AZIM, 34, 64
        bte.bte_init_mesh([bte.bte_geom(2, 3, 2, 1, 1e-8, 1e-8, 1e-8)], o)
    assert e.value.code == -1


def test_no_scattering_reports_T_L_for_T_p():
    """Every beta_b = 0: I0 never enters the update and T_p is T_L."""
    g = hot_cold(W.Geometry(2, 7, 4, 1, 10e-9, 10e-9, 10e-9))
    b = W.make_bands(4, 1, 45)
    b.beta[:] = 0.0
    wl = W.Workload("ballistic", [g], W.Dirs("inplane", n_inplane=12), b, 1e-12, 6, 3)
    s = bte.Solver(wl)
    s.step(nsteps=6, ninner=3)
    p = O.Problem(g, O.dirs_for(wl.dirs), wl.bands)
    ost = p.init_state(g.T_init)
    p.run(ost, wl.dt, 6, 3)
    TL = s.T(0, bte.BTE_T_LATTICE)
    assert np.max(np.abs(TL - ost["TL"]) / ost["TL"]) <= 1e-12
    assert np.array_equal(s.T(0, bte.BTE_T_PSEUDO), TL)
    assert np.max(np.abs(s.intensity(0) - ost["I"]) / np.abs(ost["I"])) <= 1e-11
    s.close()


def test_zero_steps_leave_the_state_unchanged():
    wl = W.cfg2(9, 7)
    s = bte.Solver(wl)
    I0, T0 = s.intensity(0), s.T(0, bte.BTE_T_PSEUDO)
    rc, st = s.step(nsteps=0, ninner=5)
    assert rc == 0 and st["launches"] == 0 and st["updates"] == 0
    assert np.array_equal(s.intensity(0), I0) and np.array_equal(s.T(0, bte.BTE_T_PSEUDO), T0)
    s.close()


def test_explicit_single_cell_with_specular_walls_is_exactly_steady():
    """One cell, every wall a mirror, equilibrium start: nothing changes."""
    g = W.Geometry(2, 1, 1, 1, 10e-9, 10e-9, 10e-9)
    W.uniform_walls(g, [W.BC_SPECULAR] * 4, [0.0] * 4)
    wl = W.Workload("mirror box", [g], W.Dirs("inplane", n_inplane=16), W.make_bands(5, 2, 46), 2e-13, 10, 1)
    s = bte.Solver(wl)
    I_start = s.intensity(0)
    s.step(nsteps=10, ninner=1, scheme=bte.BTE_EXPLICIT)
    assert np.max(np.abs(s.intensity(0) - I_start) / I_start) <= 1e-14
    assert np.max(np.abs(s.T(0, bte.BTE_T_LATTICE) - 300.0)) <= 1e-12 * 300
    s.close()


def test_exact_fixup_with_32_gauss_nodes_and_110_bands():
    """The exact solve of the fix-up takes the band quadrature in chunks of at
    most 1024 (band, node) pairs: 110 bands x 32 nodes is four chunks.  A
    cold start far from equilibrium sends cells to the fix-up; T and I match
    the oracle with the same quadrature within the FP64 bar."""
    g = W.Geometry(2, 7, 5, 1, 10e-9, 10e-9, 10e-9)
    W.uniform_walls(g, [W.BC_ISOTHERMAL, W.BC_ISOTHERMAL, W.BC_SPECULAR, W.BC_DIFFUSE], [340.0, 290.0, 0.0, 0.0])
    wl = W.Workload("32 nodes", [g], W.Dirs("inplane", n_inplane=12), W.make_bands(80, 30, 44), 2e-12, 3, 4)
    assert wl.bands.nb == 110
    T0 = W.random_temperatures(g.ncells, 45, 280.0, 340.0)
    s = bte.Solver(wl, n_gauss=32, T_init=[T0])
    rc, st = s.step(nsteps=3, ninner=4)
    assert rc >= 0 and st["nonfinite"] == 0
    assert st["solve_evals"] > 0                 # the fix-up ran
    p = O.Problem(g, O.dirs_for(wl.dirs), wl.bands, ngauss=32)
    ost = p.init_state(T0)
    p.run(ost, wl.dt, 3, 4)
    for which, key in ((bte.BTE_T_LATTICE, "TL"), (bte.BTE_T_PSEUDO, "Tp")):
        assert np.max(np.abs(s.T(0, which) - ost[key]) / ost[key]) <= 1e-12, key
    assert np.max(np.abs(s.intensity(0) - ost["I"]) / np.abs(ost["I"])) <= 1e-11
    s.close()


@pytest.mark.parametrize("nb_split", [(1, 0), (2, 1)])
def test_exact_fixup_with_fewer_bands_than_cluster_ctas(nb_split):
    """The fix-up solves each cell on a cluster of four CTAs, CTA r owning the
    bands [r nbp / 4, (r + 1) nbp / 4) of the padded band count nbp.  With one
    band (nbp 2) or three (nbp 4, one padding band) some CTAs own no real band
    or none at all, yet every CTA adds all bands in the same order and
    advances the same solve.  A cold start far from equilibrium sends cells
    to the fix-up; T and I match the oracle within the FP64 bar."""
    g = W.Geometry(2, 6, 4, 1, 10e-9, 10e-9, 10e-9)
    W.uniform_walls(g, [W.BC_ISOTHERMAL, W.BC_ISOTHERMAL, W.BC_SPECULAR, W.BC_SPECULAR], [340.0, 290.0, 0.0, 0.0])
    wl = W.Workload("few bands", [g], W.Dirs("inplane", n_inplane=8), W.make_bands(nb_split[0], nb_split[1], 46),
                    2e-12, 3, 3)
    assert wl.bands.nb == sum(nb_split)
    T0 = W.random_temperatures(g.ncells, 47, 280.0, 340.0)
    s = bte.Solver(wl, T_init=[T0])
    rc, st = s.step(nsteps=3, ninner=3)
    assert rc >= 0 and st["nonfinite"] == 0
    assert st["solve_evals"] > 0                 # the fix-up ran
    p = O.Problem(g, O.dirs_for(wl.dirs), wl.bands)
    ost = p.init_state(T0)
    p.run(ost, wl.dt, 3, 3)
    for which, key in ((bte.BTE_T_LATTICE, "TL"), (bte.BTE_T_PSEUDO, "Tp")):
        assert np.max(np.abs(s.T(0, which) - ost[key]) / ost[key]) <= 1e-12, key
    assert np.max(np.abs(s.intensity(0) - ost["I"]) / np.abs(ost["I"])) <= 1e-11
    s.close()
