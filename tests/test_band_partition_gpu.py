"""Band partition (Sec. 3.3) through the C ABI on one GPU.

Each rank is a band-range handle (bte_set_band_range) that sweeps only its
bands and hands the per-cell (E_L, E_p) partials to an exchange callback
(bte_set_exchange) once per inner iteration; after the sum every rank solves
the same temperatures.  Ranks here are host threads (each with its own handle
and stream) whose exchange meets at a host barrier, or spawned processes that
sum over a gloo group with ``bte.allreduce_exchange``.  No kernel waits on
another rank: the exchange is on the host, between launches.

Checks: temperatures and each rank's intensities against the unpartitioned
oracle (rel 1e-12 in FP64; 1e-4 K in FP32), identical temperatures on every
rank, the per-rank heat fluxes summing to the unpartitioned flux, and the error
paths (no exchange, failing exchange, bad range, late range).
"""
import datetime
import multiprocessing as mp
import os
import socket
import threading

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


class ThreadExchange:
    """Sums the ranks' partials on the host; every rank gets the same totals."""

    def __init__(self, n):
        self.parts = [None] * n
        self.bar = threading.Barrier(n, timeout=120)
        self.calls = [0] * n

    def member(self, r):
        def fn(buf):
            self.calls[r] += 1
            self.parts[r] = buf.cpu()
            self.bar.wait()
            tot = self.parts[0].clone()
            for p in self.parts[1:]:
                tot += p
            self.bar.wait()
            buf.copy_(tot)
        return fn


def run_ranks(wl, ranges, nsteps, ninner, precision=bte.BTE_FP64, scheme=bte.BTE_IMPLICIT_JACOBI):
    x = ThreadExchange(len(ranges))
    solvers = [bte.Solver(wl, precision=precision, stream=torch.cuda.Stream(), band_range=r, exchange=x.member(i))
               for i, r in enumerate(ranges)]
    stats, errs = [None] * len(ranges), []

    def body(i):
        try:
            stats[i] = solvers[i].step(nsteps=nsteps, ninner=ninner, scheme=scheme)[1]
        except Exception as e:  # re-raised below
            errs.append(e)
            x.bar.abort()
    th = [threading.Thread(target=body, args=(i,)) for i in range(len(ranges))]
    for t in th:
        t.start()
    for t in th:
        t.join(timeout=600)
    assert not errs, errs
    return solvers, stats, x


def oracle_run(wl, nsteps, ninner, scheme=O.IMPLICIT):
    g = wl.geoms[0]
    p = O.Problem(g, O.dirs_for(wl.dirs), wl.bands)
    st = p.init_state(g.T_init)
    p.run(st, wl.dt, nsteps, ninner, scheme)
    return p, st


CASES = {
    # 4 bands split 1 + 3
    "cfg1": (lambda: W.cfg1(), [(0, 1), (1, 4)], 6, 5),
    # 400 directions, 55 band-polarisations split 20 + 35: both ranges end inside a padding group of 8
    "cfg2_small": (lambda: W.cfg2(12, 9), [(0, 20), (20, 55)], 2, 4),
}


@pytest.mark.parametrize("name", list(CASES))
def test_band_ranks_match_the_oracle(name):
    mk, ranges, nsteps, ninner = CASES[name]
    wl = mk()
    solvers, stats, x = run_ranks(wl, ranges, nsteps, ninner)
    p, ref = oracle_run(wl, nsteps, ninner)
    assert x.calls == [nsteps * ninner] * len(ranges)
    assert all(s["launches"] == 3 * nsteps * ninner for s in stats)   # sweep, cell solve, fix-up
    T = [(s.T(0, bte.BTE_T_PSEUDO), s.T(0, bte.BTE_T_LATTICE)) for s in solvers]
    for Tp, TL in T[1:]:
        assert np.array_equal(Tp, T[0][0]) and np.array_equal(TL, T[0][1])
    assert np.max(np.abs(T[0][0] - ref["Tp"]) / ref["Tp"]) <= 1e-12
    assert np.max(np.abs(T[0][1] - ref["TL"]) / ref["TL"]) <= 1e-12
    scale = np.max(np.abs(ref["I"]))
    for s, (lo, hi) in zip(solvers, ranges):
        assert np.max(np.abs(s.intensity(0) - ref["I"][:, :, lo:hi])) <= 1e-12 * scale
    # heat flux: the ranks' partial fluxes sum to the whole
    q_ref, qw_ref = p.flux(ref["I"])
    q = sum(s.flux(0)[0] for s in solvers)
    qw = sum(s.flux(0)[1] for s in solvers)
    assert np.max(np.abs(q - q_ref)) <= 1e-10 * np.max(np.abs(q_ref))
    assert np.max(np.abs(qw - qw_ref)) <= 1e-10 * np.max(np.abs(q_ref))
    for s in solvers:
        s.close()


def test_sweep_ordered_band_ranks_match_the_oracle():
    """The sweep-ordered scheme on band ranges: pass, per-cell partials,
    exchange, cell solve, fix-up per inner iteration."""
    mk, ranges, nsteps, ninner = CASES["cfg2_small"]
    wl = mk()
    solvers, stats, x = run_ranks(wl, ranges, nsteps, ninner, scheme=bte.BTE_IMPLICIT_GS)
    _, ref = oracle_run(wl, nsteps, ninner, O.GAUSS_SEIDEL)
    assert x.calls == [nsteps * ninner] * len(ranges)
    assert all(s["launches"] == 4 * nsteps * ninner for s in stats)   # pass, reduction, cell solve, fix-up
    for s in solvers:
        for which, key in ((bte.BTE_T_LATTICE, "TL"), (bte.BTE_T_PSEUDO, "Tp")):
            assert np.max(np.abs(s.T(0, which) - ref[key]) / ref[key]) <= 1e-12, key
    I = ref["I"]
    for s, (b0, b1) in zip(solvers, ranges):
        assert np.max(np.abs(s.intensity(0) - I[:, :, b0:b1]) / np.abs(I[:, :, b0:b1])) <= 1e-11
    for s in solvers:
        s.close()


def test_fp32_band_ranks_within_the_reduced_mode_tolerance():
    mk, ranges, nsteps, ninner = CASES["cfg2_small"]
    wl = mk()
    solvers, _, _ = run_ranks(wl, ranges, nsteps, ninner, precision=bte.BTE_FP32)
    _, ref = oracle_run(wl, nsteps, ninner)
    for s in solvers:
        assert np.max(np.abs(s.T(0, bte.BTE_T_LATTICE) - ref["TL"])) <= 1e-4
        assert np.max(np.abs(s.T(0, bte.BTE_T_PSEUDO) - ref["Tp"])) <= 1e-4
        s.close()


def test_band_range_error_paths():
    wl = W.cfg1()
    # stepping without an exchange
    s = bte.Solver(wl, band_range=(0, 2))
    with pytest.raises(bte.BTEError) as e:
        s.step(nsteps=1, ninner=1)
    assert e.value.code == -2
    # a range after device memory is in use
    with pytest.raises(bte.BTEError) as e:
        bte.bte_set_band_range(s.h, 0, 1)
    assert e.value.code == -2
    # an exchange that fails
    cb = bte.bte_set_exchange(s.h, lambda buf, n, stream: 5)
    with pytest.raises(bte.BTEError) as e:
        s.step(nsteps=1, ninner=1)
    assert e.value.code == -7
    del cb
    s.close()
    # bad ranges
    h = bte.bte_init_mesh([bte.bte_geom(2, 4, 4, 1, 1e-8, 1e-8, 1e-8)])
    b = wl.bands
    bte.bte_set_bands(h, b.omega_lo, b.omega_hi, b.vg, b.beta, b.degeneracy)
    for lo, hi in ((-1, 2), (2, 2), (3, 2), (0, 5)):
        with pytest.raises(bte.BTEError) as e:
            bte.bte_set_band_range(h, lo, hi)
        assert e.value.code == -1
    bte.bte_destroy(h)


def test_whole_range_handle_is_the_plain_handle():
    """band_range = (0, nb) stores every band: no exchange is needed and the
    result is bit-identical to a handle without a range."""
    wl = W.cfg1()
    a = bte.Solver(wl)
    b = bte.Solver(wl, band_range=(0, wl.bands.nb))
    a.step(nsteps=3, ninner=4)
    b.step(nsteps=3, ninner=4)
    assert np.array_equal(a.intensity(0), b.intensity(0))
    assert np.array_equal(a.T(0, bte.BTE_T_PSEUDO), b.T(0, bte.BTE_T_PSEUDO))
    a.close(); b.close()


# ---- ranks as processes over a gloo group ---------------------------------
def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _proc_rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    try:
        dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=120))
        mk, ranges, nsteps, ninner = CASES["cfg1"]
        wl = mk()
        s = bte.Solver(wl, band_range=ranges[rank], exchange=bte.allreduce_exchange())
        s.step(nsteps=nsteps, ninner=ninner)
        q.put((rank, "ok", s.T(0, bte.BTE_T_PSEUDO), s.T(0, bte.BTE_T_LATTICE), s.intensity(0)))
        s.close()
    except Exception as e:
        q.put((rank, "error", repr(e), None, None))
    finally:
        if dist.is_initialized():
            dist.destroy_process_group()


def test_band_ranks_as_processes_over_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_proc_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = {}
    try:
        for _ in range(2):
            r = q.get(timeout=600)
            out[r[0]] = r[1:]
    finally:
        for p in procs:
            p.join(timeout=120)
            if p.is_alive():
                p.kill()
    assert all(out[r][0] == "ok" for r in out), out
    mk, ranges, nsteps, ninner = CASES["cfg1"]
    wl = mk()
    _, ref = oracle_run(wl, nsteps, ninner)
    assert np.array_equal(out[0][1], out[1][1])
    assert np.max(np.abs(out[0][1] - ref["Tp"]) / ref["Tp"]) <= 1e-12
    assert np.max(np.abs(out[0][2] - ref["TL"]) / ref["TL"]) <= 1e-12
    scale = np.max(np.abs(ref["I"]))
    for r, (lo, hi) in enumerate(ranges):
        assert np.max(np.abs(out[r][3] - ref["I"][:, :, lo:hi])) <= 1e-12 * scale


def test_band_ranks_with_diffuse_and_partially_specular_walls():
    """Wall ghosts of a rank's own bands (diffuse rows, per-direction partial
    rows) under the band partition, against the oracle's whole-band run."""
    def mk():
        wl = W.cfg2(12, 9)
        wl.geoms[0].bc[2] = (W.BC_DIFFUSE, None)
        wl.geoms[0].bc[3] = (W.BC_PARTIAL, 0.3)
        return wl
    wl = mk()
    ranges = [(0, 20), (20, 55)]
    solvers, stats, x = run_ranks(wl, ranges, 2, 4)
    _, ref = oracle_run(mk(), 2, 4)
    for s in solvers:
        assert np.max(np.abs(s.T(0, bte.BTE_T_LATTICE) - ref["TL"]) / ref["TL"]) <= 1e-12
    I = ref["I"]
    for s, (b0, b1) in zip(solvers, ranges):
        assert np.max(np.abs(s.intensity(0) - I[:, :, b0:b1]) / np.abs(I[:, :, b0:b1])) <= 1e-11
    for s in solvers:
        s.close()
