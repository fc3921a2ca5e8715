"""Band partition (Sec. 3.3) on host ranks: world_size-2 gloo processes.

The bands couple only through the temperature step, which needs per-cell sums
over every band.  Each rank runs the oracle's time loop over its own band range
and sums the per-cell (E_L, E_p) partials with the library's exchange helper
(``bte.allreduce_exchange``, a gloo all-reduce here).  The ranks' results must
equal the unpartitioned oracle run (up to the order of the band sum), and every
rank must hold the same temperatures bit for bit.  A rank that fails inside the
exchange must surface as an error on every rank, not as a hang.
"""
import datetime
import multiprocessing as mp
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist

from oracle import oracle as O
from paper_2305_19400_gb300 import bte, workloads as W


@pytest.fixture(scope="module", autouse=True)
def _built():
    O.build()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _case(name):
    if name == "cfg1":
        wl = W.cfg1()
        return wl, [(0, 1), (1, 4)], 10, 5
    wl = W.cfg2(10, 8)                       # 400 directions, 55 band-polarisations
    return wl, [(0, 27), (27, 55)], 2, 4


def _rank_main(rank, world, port, name, fail_at, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), OMP_NUM_THREADS="2")
    try:
        dist.init_process_group("gloo", rank=rank, world_size=world,
                                timeout=datetime.timedelta(seconds=8 if fail_at else 120))
        wl, ranges, nsteps, ninner = _case(name)
        lo, hi = ranges[rank]
        g = wl.geoms[0]
        p = O.Problem(g, O.dirs_for(wl.dirs), wl.bands)
        st = p.init_state(g.T_init)
        xch = bte.allreduce_exchange()
        calls = [0]

        def total(E):
            calls[0] += 1
            if fail_at and rank == 1 and calls[0] == fail_at:
                raise RuntimeError("rank 1 drops out of the exchange")
            t = torch.from_numpy(np.ascontiguousarray(E))
            xch(t)
            return t.numpy()
        p.run_bands(st, lo, hi, total, wl.dt, nsteps, ninner)
        q.put((rank, "ok", st["I"][:, :, lo:hi].copy(), st["Tp"].copy(), st["TL"].copy(), calls[0]))
    except Exception as e:  # reported to the parent; the process still exits cleanly
        q.put((rank, "error", repr(e), None, None, None))
    finally:
        if dist.is_initialized():
            try:
                dist.destroy_process_group()
            except Exception:
                pass


def _run_ranks(name, fail_at=0, world=2):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, name, fail_at, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = {}
    try:
        for _ in range(world):
            r = q.get(timeout=300)
            out[r[0]] = r[1:]
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.kill()
    return out


@pytest.mark.parametrize("name", ["cfg1", "cfg2_small"])
def test_band_ranks_match_the_unpartitioned_run(name):
    out = _run_ranks(name)
    assert all(out[r][0] == "ok" for r in out), out
    wl, ranges, nsteps, ninner = _case(name)
    g = wl.geoms[0]
    p = O.Problem(g, O.dirs_for(wl.dirs), wl.bands)
    ref = p.init_state(g.T_init)
    p.run(ref, wl.dt, nsteps, ninner)
    # every rank solved the same temperatures from the same exchanged sums
    assert np.array_equal(out[0][2], out[1][2]) and np.array_equal(out[0][3], out[1][3])
    assert out[0][4] == out[1][4] == nsteps * ninner          # one exchange per inner iteration
    for key, k in (("Tp", 2), ("TL", 3)):
        assert np.max(np.abs(out[0][k] - ref[key]) / ref[key]) <= 1e-12, key
    scale = np.max(np.abs(ref["I"]))
    for r, (lo, hi) in enumerate(ranges):
        assert np.max(np.abs(out[r][1] - ref["I"][:, :, lo:hi])) <= 1e-12 * scale
    # the transient actually moved the temperatures (the comparison is not of an unchanged state)
    assert np.max(np.abs(ref["TL"] - g.T_init)) > 1e-4


def test_a_rank_failing_in_the_exchange_is_an_error_on_every_rank():
    out = _run_ranks("cfg1", fail_at=3)
    # the failing rank's callback error ends its run; the survivor's all-reduce
    # ends with an error when the peer leaves, not with a hang
    assert out[1][0] == "error" and "band-sum callback failed" in out[1][1]
    assert out[0][0] == "error"


def test_allreduce_exchange_sums_host_tensors_in_place():
    """The exchange helper on a one-rank gloo group is the identity on the buffer."""
    port = _free_port()
    store = dist.TCPStore("127.0.0.1", port, 1, True, timeout=datetime.timedelta(seconds=30))
    dist.init_process_group("gloo", store=store, rank=0, world_size=1)
    try:
        buf = torch.arange(10, dtype=torch.float64)
        before = buf.data_ptr()
        bte.allreduce_exchange()(buf)
        assert buf.data_ptr() == before and torch.equal(buf, torch.arange(10, dtype=torch.float64))
    finally:
        dist.destroy_process_group()
