"""Batched geometries in one persistent launch, CUDA-graph replay and the
autotuner: each must leave the arithmetic of every cell unchanged, so results
are compared bitwise with the plain path; the batch is also checked against
the FP64 oracle per geometry."""
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


def _subset(wl, idx):
    return W.Workload(wl.name + "_sub", [wl.geoms[i] for i in idx], wl.dirs, wl.bands, wl.dt, wl.nsteps, wl.ninner,
                      wl.precision)


@pytest.mark.parametrize("precision", [bte.BTE_FP32, bte.BTE_FP64])
def test_batched_geometries_equal_single_runs_bitwise(precision):
    full = W.cfg5()
    wl = _subset(full, [6, 10, 4, 7])          # sizes 41x42, 35x38, 98x61, 39x60 (ragged tiles)
    batch = bte.Solver(wl, precision=precision, use_graph=True)
    batch.step(nsteps=2, ninner=4)
    for gi, g in enumerate(wl.geoms):
        one = bte.Solver(_subset(wl, [gi]), precision=precision)
        one.step(nsteps=2, ninner=4)
        assert np.array_equal(batch.T(gi, bte.BTE_T_PSEUDO), one.T(0, bte.BTE_T_PSEUDO)), gi
        assert np.array_equal(batch.intensity(gi), one.intensity(0)), gi
        one.close()
    batch.close()


def test_batch_matches_oracle_per_geometry_fp32():
    full = W.cfg5()
    wl = _subset(full, [10, 6])
    s = bte.Solver(wl, precision=bte.BTE_FP32, use_graph=True, autotune=True)
    s.step(nsteps=2, ninner=4)
    for gi, g in enumerate(wl.geoms):
        p = O.Problem(g, O.dirs_for(wl.dirs), wl.bands)
        st = p.init_state(g.T_init)
        p.run(st, wl.dt, 2, 4)
        assert np.max(np.abs(s.T(gi, bte.BTE_T_LATTICE) - st["TL"])) <= 1e-4
        assert np.max(np.abs(s.T(gi, bte.BTE_T_PSEUDO) - st["Tp"])) <= 1e-4
        assert st["TL"].max() - 300.0 > 1e-3
    s.close()


def test_graph_replay_equals_eager_launches_bitwise():
    wl = W.cfg2(24, 17)
    eager = bte.Solver(wl)
    graph = bte.Solver(wl, use_graph=True)
    for nsteps, ninner in ((1, 5), (2, 5), (1, 4), (3, 5)):   # different buffer rotations and graph keys
        r1 = eager.step(nsteps=nsteps, ninner=ninner)[1]
        r2 = graph.step(nsteps=nsteps, ninner=ninner)[1]
        assert r1["launches"] == r2["launches"] == 2 * nsteps * ninner   # sweep + fix-up
    assert np.array_equal(eager.intensity(0), graph.intensity(0))
    assert np.array_equal(eager.T(0, bte.BTE_T_PSEUDO), graph.T(0, bte.BTE_T_PSEUDO))
    eager.close(); graph.close()


def test_autotune_reports_candidates_and_keeps_results():
    """Cells per CTA, grid and register variant leave every result bit for bit
    the same; a different number of directions per team step regroups each
    lane's direction sums, which changes results at the rounding level only."""
    wl = W.cfg2(40, 33)
    plain = bte.Solver(wl)
    tuned = bte.Solver(wl)
    rep = bte.bte_autotune(tuned.h, wl.dt)
    lines = [l for l in rep.strip().splitlines()]
    assert lines[0].startswith("cells_per_cta") and lines[-1].startswith("chosen")
    assert lines[0].split(",")[-1] == "directions_per_step"
    cands = [l.split(",") for l in lines[1:-1]]
    dteams = sorted({int(c[5]) for c in cands})
    assert dteams == [1, 2]                  # the default (2 for 400 FP64 rows of 56 bands) and half of it
    default_dteam, chosen_dteam = int(cands[0][5]), int(lines[-1].split(",")[5])
    assert default_dteam == 2 and chosen_dteam in dteams
    for _ in range(2):
        plain.step(nsteps=2, ninner=5)
        tuned.step(nsteps=2, ninner=5)
    Ip, It = plain.intensity(0), tuned.intensity(0)
    Tp_, Tt = plain.T(0, bte.BTE_T_LATTICE), tuned.T(0, bte.BTE_T_LATTICE)
    if chosen_dteam == default_dteam:
        assert np.array_equal(Ip, It) and np.array_equal(Tp_, Tt)
    else:
        assert np.max(np.abs(It - Ip) / np.abs(Ip)) <= 1e-13
        assert np.max(np.abs(Tt - Tp_) / Tp_) <= 1e-13
    plain.close(); tuned.close()


def test_graph_replay_survives_a_dt_change():
    wl = W.cfg2(10, 9)
    a = bte.Solver(wl, use_graph=True)
    b = bte.Solver(wl)
    for dt in (1e-12, 2e-12, 1e-12):
        a.step(nsteps=1, ninner=3, dt=dt)
        b.step(nsteps=1, ninner=3, dt=dt)
    assert np.array_equal(a.intensity(0), b.intensity(0))
    a.close(); b.close()
