"""Reduced-precision storage modes against the FP64 CPU oracle.

FP32 and BF16 store the deviation I - I0_b(T_ref) and run the sweep in FP32;
the reduction, temperature solve and I0 stay FP64.  Targets (FP32): max |dT|
<= 1e-4 K on T_L and T_p, relative heat-flux error (2-norm over all cells and
axes) <= 1e-5.  BF16 is reported with a looser bound.  The errors are printed
so a run log records them.
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


def _errors(wl, precision, nsteps, ninner, T_init=None):
    s = bte.Solver(wl, precision=precision, T_init=None if T_init is None else [T_init])
    rc, st = s.step(nsteps=nsteps, ninner=ninner)
    TL, Tp = s.T(0, bte.BTE_T_LATTICE), s.T(0, bte.BTE_T_PSEUDO)
    q, qw = s.flux(0)
    I = s.intensity(0)
    s.close()
    g = wl.geoms[0]
    p = O.Problem(g, O.dirs_for(wl.dirs), wl.bands)
    ost = p.init_state(g.T_init if T_init is None else T_init)
    p.run(ost, wl.dt, nsteps, ninner)
    q_ref, qw_ref = p.flux(ost["I"])
    err = {
        "dT_L": float(np.max(np.abs(TL - ost["TL"]))),
        "dT_p": float(np.max(np.abs(Tp - ost["Tp"]))),
        "q_rel": float(np.linalg.norm(q - q_ref) / np.linalg.norm(q_ref)),
        "q_wall_rel": float(np.max(np.abs(qw - qw_ref)) / np.max(np.abs(qw_ref))),
        "I_rel_max": float(np.max(np.abs(I - ost["I"]) / np.abs(ost["I"]))),
        "heating_K": float(ost["TL"].max() - ost["TL"].min()),
        "evals_per_solve": st["solve_evals"] / max(st["solves"], 1),
    }
    return err


def _cfg3_small(n=16):
    wl = W.cfg3(n)
    return wl


@pytest.mark.parametrize("n,nsteps", [(16, 3)])
def test_fp32_3d_subsample_meets_the_stated_tolerance(n, nsteps):
    wl = _cfg3_small(n)
    e = _errors(wl, bte.BTE_FP32, nsteps, 15)
    print("FP32 3-D", n, "cube:", e)
    assert e["heating_K"] > 1e-3
    assert e["dT_L"] <= 1e-4 and e["dT_p"] <= 1e-4, e
    assert e["q_rel"] <= 1e-5 and e["q_wall_rel"] <= 1e-5, e


def test_fp32_2d_hot_spot_grid_meets_the_stated_tolerance():
    wl = W.cfg2(19, 13)
    e = _errors(wl, bte.BTE_FP32, 4, 15)
    print("FP32 2-D 19x13:", e)
    assert e["dT_L"] <= 1e-4 and e["dT_p"] <= 1e-4, e
    assert e["q_rel"] <= 1e-5 and e["q_wall_rel"] <= 1e-5, e


def test_bf16_storage_error_is_reported():
    wl = W.cfg2(19, 13)
    e = _errors(wl, bte.BTE_BF16, 4, 15)
    print("BF16 2-D 19x13:", e)
    assert e["dT_L"] <= 0.05 and e["dT_p"] <= 0.05, e


def test_fp32_uniform_equilibrium_at_the_reference_temperature_is_exact():
    wl = W.cfg2(12, 9)
    g = wl.geoms[0]
    g.bc = [(W.BC_ISOTHERMAL, np.full(g.ny, 300.0)), (W.BC_ISOTHERMAL, np.full(g.ny, 300.0)),
            (W.BC_SPECULAR, None), (W.BC_SPECULAR, None)]
    for prec in (bte.BTE_FP32, bte.BTE_BF16):
        s = bte.Solver(wl, precision=prec)
        s.step(nsteps=3, ninner=5)
        assert np.max(np.abs(s.T(0, bte.BTE_T_PSEUDO) - 300.0)) <= 1e-12 * 300
        assert np.max(np.abs(s.T(0, bte.BTE_T_LATTICE) - 300.0)) <= 1e-12 * 300
        s.close()


def test_fp32_explicit_scheme_and_multi_geometry():
    geoms = []
    for nx, ny, th in ((7, 5, 312.0), (4, 9, 306.0)):
        g = W.Geometry(2, nx, ny, 1, 10e-9, 10e-9, 10e-9)
        W.uniform_walls(g, [W.BC_ISOTHERMAL, W.BC_ISOTHERMAL, W.BC_SPECULAR, W.BC_SPECULAR], [th, 300.0, 0, 0])
        geoms.append(g)
    wl = W.Workload("pair", geoms, W.Dirs("inplane", n_inplane=16), W.make_bands(40, 15, 19405), 2e-13, 30, 1)
    s = bte.Solver(wl, precision=bte.BTE_FP32)
    s.step(scheme=bte.BTE_EXPLICIT)
    for gi, g in enumerate(geoms):
        p = O.Problem(g, O.dirs_for(wl.dirs), wl.bands)
        ost = p.init_state(g.T_init)
        p.run(ost, wl.dt, wl.nsteps, 1, O.EXPLICIT)
        assert np.max(np.abs(s.T(gi, bte.BTE_T_LATTICE) - ost["TL"])) <= 1e-4
    s.close()


def test_fp32_state_round_trip_through_fp64_host_buffers():
    wl = W.cfg2(9, 7)
    a = bte.Solver(wl, precision=bte.BTE_FP32)
    a.step(nsteps=2, ninner=4)
    I, Tp = a.intensity(0), a.T(0, bte.BTE_T_PSEUDO)
    b = bte.Solver(wl, precision=bte.BTE_FP32)
    bte.bte_set_intensity(b.h, 0, I, Tp)
    # the restored FP32 deviations are the same floats, so the fields agree to FP32 rounding of I0_ref + dI
    assert np.max(np.abs(b.intensity(0) - I) / np.abs(I)) <= 1e-15
    a.step(nsteps=1, ninner=4)
    b.step(nsteps=1, ninner=4)
    assert np.max(np.abs(a.T(0, bte.BTE_T_LATTICE) - b.T(0, bte.BTE_T_LATTICE))) <= 1e-9
    a.close(); b.close()


def test_fp32_deviation_storage_stays_accurate_over_a_long_run():
    """400 steps x 15 inner iterations (6000 sweeps) of the 400-direction
    workload on a 32x24 grid: FP32 storage against the FP64 path (itself at
    rel 1e-12 of the oracle) stays within 1e-5 K on T_L and 1e-5 on the heat
    flux; the error grows about linearly (1e-6 K measured at 400 steps)."""
    wl = W.cfg2(32, 24)
    a = bte.Solver(wl, precision=bte.BTE_FP64, use_graph=True)
    b = bte.Solver(wl, precision=bte.BTE_FP32, use_graph=True)
    for s in (a, b):
        s.step(nsteps=400, ninner=15, want_stats=False)
    T64 = a.T(0, bte.BTE_T_LATTICE)
    assert T64.max() - 300.0 > 5.0                       # the hot wall heated the grid
    assert np.max(np.abs(b.T(0, bte.BTE_T_LATTICE) - T64)) <= 1e-5
    q64, _ = a.flux(0)
    q32, _ = b.flux(0)
    assert np.linalg.norm(q32 - q64) / np.linalg.norm(q64) <= 1e-5
    a.close()
    b.close()
