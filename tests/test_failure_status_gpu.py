"""Failure statuses of bte_step, triggered from the host without faulting the GPU.

* BTE_E_NONFINITE: a checkpoint restore (bte_set_intensity) carrying a NaN
  row in one cell; the next step's per-cell energy of that cell is not finite
  and the call says so.  Restoring finite data makes the handle step again.
* BTE_W_FALLBACK: learned mode with deliberately wrong network weights (net A
  answers 1.5 K for every energy, net B is flat).  The networks start the
  exact solve of cells whose cached temperature model has no usable root; a
  checkpoint restore that claims T_p = 1 K for a 300 K field makes that so
  for every cell (the model at 1 K puts its root far above 5000 K).  From
  the 1.5 K guess the Halley step leaves [1, 5000] K and the solve falls back
  to bisection.  The call reports the fallbacks, and the temperatures still
  equal the FP64 oracle's (same restore, same step) to rel 1e-12, because
  bisection runs to the same root.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import mlp as M
from oracle import oracle as O
from paper_2305_19400_gb300 import bte, workloads as W

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2305_19400_gb300 import build as B
    B.build()
    O.build()


@pytest.mark.parametrize("precision", [bte.BTE_FP64, bte.BTE_FP32])
def test_nan_intensity_row_returns_nonfinite_and_the_handle_recovers(precision):
    wl = W.cfg2(7, 5)
    s = bte.Solver(wl, precision=precision)
    s.step(nsteps=1, ninner=3)
    I = s.intensity(0)
    Tp = s.T(0, bte.BTE_T_PSEUDO)
    bad = I.copy()
    bad[11, 5:9, :] = np.nan
    bte.bte_set_intensity(s.h, 0, bad, Tp)
    with pytest.raises(bte.BTEError) as e:
        s.step(nsteps=1, ninner=2)
    assert e.value.code == bte.BTE_E_NONFINITE and "non-finite" in str(e.value)
    # a finite restore makes the handle step normally again
    bte.bte_set_intensity(s.h, 0, I, Tp)
    rc, st = s.step(nsteps=1, ninner=2)
    assert rc == 0 and st["nonfinite"] == 0
    assert np.all(np.isfinite(s.T(0, bte.BTE_T_LATTICE)))
    s.close()


def _wrong_nets(wl, T_lo, T_hi, T_guess):
    """Net A: every weight 0 and the output bias chosen so that the guess is
    T_guess for any energy; net B: all zero (a flat surrogate, whose Newton
    step is refused)."""
    pa = np.zeros(M.n_params(1), dtype=np.float32)
    pa[-1] = 2.0 * (T_guess - T_lo) / (T_hi - T_lo) - 1.0
    pb = np.zeros(M.n_params(wl.bands.nb), dtype=np.float32)
    return pa, pb


def test_wrong_network_weights_fall_back_to_bisection_with_unchanged_results():
    wl = W.cfg2(13, 9)
    g = wl.geoms[0]
    s = bte.Solver(wl, learned=True)
    bte.bte_train_mlp(s.h, 1 << 14, 250.0, 400.0, 1, seed=3)
    pa, pb = _wrong_nets(wl, 250.0, 400.0, 1.5)
    bte.bte_mlp_set_params(s.h, 0, pa)
    bte.bte_mlp_set_params(s.h, 1, pb)
    # restore the 300 K field with T_p = 1 K: no cell keeps a usable model root
    p = O.Problem(g, O.dirs_for(wl.dirs), wl.bands)
    ost = p.init_state(g.T_init)
    Tp1 = np.full(g.ncells, 1.0)
    bte.bte_set_intensity(s.h, 0, ost["I"], Tp1)
    rc, st = s.step(nsteps=1, ninner=3)
    assert rc == bte.BTE_W_FALLBACK and st["fallbacks"] > 0, (rc, st)
    ost["Tp"] = Tp1.copy()
    ost["I0"] = np.tile(O.I0(wl.bands, 1.0)[0], (g.ncells, 1))
    p.run(ost, wl.dt, 1, 3)
    for which, key in ((bte.BTE_T_LATTICE, "TL"), (bte.BTE_T_PSEUDO, "Tp")):
        assert np.max(np.abs(s.T(0, which) - ost[key]) / ost[key]) <= 1e-12
    # the same wrong start through the batch solve: every root still exact
    T_true = W.random_temperatures(64, 41, 280.0, 330.0)
    a = 4 * np.pi * wl.bands.beta / wl.bands.vg
    Ep = np.array([float(np.dot(a, O.I0(wl.bands, t)[0])) for t in T_true])
    T, ev = bte.bte_solve_T(s.h, Ep, learned=True)
    assert np.max(np.abs(T - T_true) / T_true) <= 1e-12
    assert ev.min() > 10   # bisection: tens of evaluations, not Halley's handful
    s.close()
