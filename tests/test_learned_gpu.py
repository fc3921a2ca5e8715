"""The learned temperature / equilibrium guess (nets A and B) on the GPU.

* gradients of the CUDA training kernels against the oracle's FP64 backprop;
* training on device-generated pairs reaches a small loss;
* the learned start + exact FP64 refinement solves the T_p equation to the
  same root as the oracle, and the test reports (and bounds) what the guess
  saves in exact quadrature evaluations against a cold start, next to a warm
  start;
* a learned-mode run of the hot path matches the oracle like the plain mode.
"""
import math

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


@pytest.fixture(scope="module")
def trained():
    wl = W.cfg2(6, 5)
    s = bte.Solver(wl, learned=True)
    loss = bte.bte_train_mlp(s.h, 1 << 18, 250.0, 400.0, 6, seed=11)
    yield wl, s, loss
    s.close()


@pytest.mark.parametrize("net", [0, 1])
def test_gpu_gradients_match_oracle_backprop(net):
    wl = W.cfg2(4, 3)
    s = bte.Solver(wl)
    k = 1 if net == 0 else wl.bands.nb
    rng = np.random.default_rng(20 + net)
    p = rng.normal(0.0, 0.25, M.n_params(k)).astype(np.float32)
    bte.bte_mlp_set_params(s.h, net, p)
    x = rng.uniform(-1, 1, 512).astype(np.float32)
    y = rng.uniform(-1, 1, (k, 512)).astype(np.float32)
    g, loss = bte.bte_mlp_grad(s.h, net, x, y)
    loss_ref, g_ref = M.loss_and_grad(p.astype(np.float64), k, x.astype(np.float64), y.astype(np.float64))
    assert abs(loss - loss_ref) <= 1e-5 * loss_ref
    # per parameter tensor: relative error of the gradient in the 2-norm
    sizes = [64, 64, 64 * 64, 64, k * 64, k]
    o = 0
    for n in sizes:
        a, b = g[o:o + n].astype(np.float64), g_ref[o:o + n]
        assert np.linalg.norm(a - b) <= 1e-4 * np.linalg.norm(b), (net, o, np.linalg.norm(a - b) / np.linalg.norm(b))
        o += n
    s.close()


def test_training_on_the_device_reaches_a_small_loss(trained):
    wl, s, loss = trained
    print("training loss (normalised MSE) net A, net B:", loss)
    assert loss[0] < 2e-4 and loss[1] < 5e-4   # 1536 Adam steps on 2^18 pairs


def _energies(wl, T):
    Wt = 4 * math.pi
    a = Wt * wl.bands.beta / wl.bands.vg
    return np.array([float(np.dot(a, O.I0(wl.bands, t)[0])) for t in T])


def test_learned_start_solves_to_the_oracle_root_and_saves_evaluations(trained):
    wl, s, _ = trained
    T_true = W.random_temperatures(200, 31, 260.0, 390.0)
    Ep = _energies(wl, T_true)
    T_cold, ev_cold = bte.bte_solve_T(s.h, Ep, np.full(200, 300.0))
    T_learn, ev_learn = bte.bte_solve_T(s.h, Ep, learned=True)
    T_warm, ev_warm = bte.bte_solve_T(s.h, Ep, T_true * (1 + 1e-6))
    for T in (T_cold, T_learn, T_warm):
        assert np.max(np.abs(T - T_true) / T_true) <= 1e-12
    print("mean exact evaluations per solve: cold start 300 K %.2f, learned %.2f, warm start (1e-6 off) %.2f"
          % (ev_cold.mean(), ev_learn.mean(), ev_warm.mean()))
    assert ev_learn.mean() < ev_cold.mean()
    assert ev_warm.mean() <= ev_learn.mean()


@pytest.mark.parametrize("precision,tol", [(bte.BTE_FP64, "rel1e-12"), (bte.BTE_FP32, "abs1e-4")])
def test_learned_mode_run_matches_the_oracle(precision, tol):
    wl = W.cfg2(13, 9)
    s = bte.Solver(wl, precision=precision, learned=True)
    bte.bte_train_mlp(s.h, 1 << 16, 250.0, 400.0, 3, seed=5)
    rc, st = s.step(nsteps=3, ninner=6)
    g = wl.geoms[0]
    p = O.Problem(g, O.dirs_for(wl.dirs), wl.bands)
    ost = p.init_state(g.T_init)
    p.run(ost, wl.dt, 3, 6)
    for which, key in ((bte.BTE_T_LATTICE, "TL"), (bte.BTE_T_PSEUDO, "Tp")):
        d = np.abs(s.T(0, which) - ost[key])
        if tol == "rel1e-12":
            assert np.max(d / ost[key]) <= 1e-12
        else:
            assert np.max(d) <= 1e-4
    s.close()


def test_learned_mode_requires_training():
    wl = W.cfg2(4, 4)
    s = bte.Solver(wl, learned=True)
    with pytest.raises(bte.BTEError) as e:
        s.step(nsteps=1, ninner=1)
    assert e.value.code == -2
    s.close()
