"""The learned 3-D workload and the 48-geometry batch against the FP64 oracle,
at the sizes the oracle finishes in seconds and in the launch configuration
the benchmark times (FP32 deviation storage, CUDA graph, autotuned shape).

* Learned workload (3-D, 400 directions, 55 band-pols, x walls 300 / 305 K,
  mirror y and z walls, FP32 + learned guess): a 20 x 20 x 10 grid, 4 time
  steps x 15 inner iterations, networks trained on the GPU on 1e6 pairs over
  [250, 400] K as in the benchmark; and the learned temperature solve on 1e5
  random cells (energies from the oracle's band quadrature at known
  temperatures), Newton-level, against those temperatures and the oracle's own
  solve.
* Batch (48 seeded 2-D geometries of uneven size, FP32, one persistent launch
  per inner iteration): the smallest, the largest and two geometries drawn at
  random (SplitMix64 seed 19405 + 1000), each on its whole grid, 2 time steps
  x 12 inner iterations, against the oracle run of that geometry alone.

Targets (the reduced modes' contract): max |dT| <= 1e-4 K for T_L and T_p,
heat flux within 1e-5 relative (2-norm over the cells, and per wall relative
to the largest wall flux)."""
import gc
import math

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


def _free_device_memory():
    gc.collect()
    torch.cuda.synchronize()
    torch.cuda.empty_cache()


def _compare(s, gi, wl, g, nsteps, ninner):
    p = O.Problem(g, O.dirs_for(wl.dirs), wl.bands)
    ost = p.init_state(g.T_init)
    p.run(ost, wl.dt, nsteps, ninner)
    dTL = float(np.max(np.abs(s.T(gi, bte.BTE_T_LATTICE) - ost["TL"])))
    dTp = float(np.max(np.abs(s.T(gi, bte.BTE_T_PSEUDO) - ost["Tp"])))
    q, qw = s.flux(gi)
    q_ref, qw_ref = p.flux(ost["I"])
    eq = float(np.linalg.norm(q - q_ref) / np.linalg.norm(q_ref))
    ew = float(np.max(np.abs(qw - qw_ref)) / np.max(np.abs(qw_ref)))
    return dTL, dTp, eq, ew, ost


def test_learned_3d_20x20x10_fp32_graph_matches_the_oracle():
    _free_device_memory()
    wl = W.cfg4(20, 20, 10, nsteps=4, ninner=15)
    s = bte.Solver(wl, precision=bte.BTE_FP32, use_graph=True, learned=True)
    loss = bte.bte_train_mlp(s.h, 1_000_000, 250.0, 400.0, 4, seed=1)
    bte.bte_autotune(s.h, wl.dt)
    rc, st = s.step()
    assert rc in (0, bte.BTE_W_FALLBACK) and st["nonfinite"] == 0
    dTL, dTp, eq, ew, ost = _compare(s, 0, wl, wl.geoms[0], wl.nsteps, wl.ninner)
    print(f"learned 3-D 20x20x10, 4 x 15: max|dT_L| {dTL:.2e} K, max|dT_p| {dTp:.2e} K, cell flux {eq:.2e}, "
          f"wall flux {ew:.2e}; training loss {loss}; solves {st['solves']}, evaluations {st['solve_evals']}")
    assert dTL <= 1e-4 and dTp <= 1e-4
    assert eq <= 1e-5 and ew <= 1e-5
    # the heat has entered from the hot +x wall
    assert ost["TL"].max() > 300.01
    s.close()


def test_learned_solve_on_1e5_random_cells_matches_the_oracle_roots():
    _free_device_memory()
    wl = W.cfg4(4, 4, 2)
    s = bte.Solver(wl, precision=bte.BTE_FP32, learned=True)
    bte.bte_train_mlp(s.h, 1_000_000, 250.0, 400.0, 4, seed=1)
    n = 100_000
    T_true = W.random_temperatures(n, 19404, 250.0, 400.0)
    a = 4 * math.pi * wl.bands.beta / wl.bands.vg
    Ep = np.array([float(np.dot(a, O.I0(wl.bands, t)[0])) for t in T_true])
    T_l, ev_l = bte.bte_solve_T(s.h, Ep, learned=True)
    T_c, ev_c = bte.bte_solve_T(s.h, Ep, np.full(n, 300.0))
    rel_l = float(np.max(np.abs(T_l - T_true) / T_true))
    rel_c = float(np.max(np.abs(T_c - T_true) / T_true))
    # the oracle's own Newton solve on a sample of the same energies
    g = wl.geoms[0]
    p = O.Problem(g, O.dirs_for(wl.dirs), wl.bands)
    idx = np.arange(0, n, 97)
    T_o = np.array([p.solve_T(a, float(Ep[i]), 300.0)[0] for i in idx])
    rel_o = float(np.max(np.abs(T_l[idx] - T_o) / T_o))
    print(f"1e5 cells: learned start max rel err {rel_l:.1e} ({ev_l.mean():.2f} evaluations per solve), "
          f"cold start {rel_c:.1e} ({ev_c.mean():.2f}); against the oracle's Newton on {idx.size} cells {rel_o:.1e}")
    assert rel_l <= 1e-12 and rel_c <= 1e-12 and rel_o <= 1e-12
    assert ev_l.mean() < ev_c.mean()
    s.close()


def _batch_picks(wl):
    cells = [g.ncells for g in wl.geoms]
    picks = [int(np.argmin(cells)), int(np.argmax(cells))]
    rng = W.SplitMix64(19405 + 1000)
    while len(picks) < 4:
        k = rng.randint(0, len(cells) - 1)
        if k not in picks:
            picks.append(k)
    return picks


def test_batch_of_48_geometries_matches_the_oracle_on_four_whole_geometries():
    _free_device_memory()
    wl = W.cfg5(nsteps=2, ninner=12)
    s = bte.Solver(wl, precision=bte.BTE_FP32, use_graph=True)
    bte.bte_autotune(s.h, wl.dt)
    rc, st = s.step()
    assert rc in (0, bte.BTE_W_FALLBACK) and st["nonfinite"] == 0
    for gi in _batch_picks(wl):
        g = wl.geoms[gi]
        dTL, dTp, eq, ew, _ = _compare(s, gi, wl, g, wl.nsteps, wl.ninner)
        print(f"batch geometry {gi} ({g.nx}x{g.ny}, hot wall {g.bc[0][1][0]:.2f} K): max|dT_L| {dTL:.2e} K, "
              f"max|dT_p| {dTp:.2e} K, cell flux {eq:.2e}, wall flux {ew:.2e}")
        assert dTL <= 1e-4 and dTp <= 1e-4
        assert eq <= 1e-5 and ew <= 1e-5
    s.close()
    del s
    _free_device_memory()
