"""Partially specular walls (bte_set_specularity) through the C ABI against the
FP64 oracle.

A side with specularity p gives every incoming direction p x the wall cell's
mirrored value + (1 - p) x its diffuse value.  Checks: FP64 parity (rel 1e-12
on T, 1e-11 on I) with point-Jacobi and sweep-ordered inner iterations, the
p = 1 and p = 0 limits against mirror and diffuse walls, FP32 in 3-D within
1e-4 K, BF16 within its reported error, zero net flux through the walls, and
graph replay, including a specularity changed after a capture.
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
