"""bench.py with N > 1 ranks runs the band partition (Sec. 3.3) by default.

Two ranks launched by torch.distributed.run share the one GPU of this machine and
exchange their per-cell energy partials over gloo (the exchange is a host
all-reduce between launches; no kernel waits on another rank).  The test
checks the JSON line rank 0 prints (the band split, strong scaling, the
roofline from the sweeps' own event timing) and that the temperatures after
the first step equal those of the unpartitioned single-rank run."""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SMALL = ["--nx", "24", "--ny", "16", "--steps", "2", "--warmup", "3", "--no-variants", "--no-cpu-baseline"]


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2305_19400_gb300 import build as B
    B.build()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _json_line(out):
    lines = [ln for ln in out.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, out[-3000:]
    return json.loads(lines[0])


def test_two_ranks_split_the_bands_and_match_the_single_rank_run(tmp_path):
    t1, t2 = str(tmp_path / "single.npy"), str(tmp_path / "parted.npy")
    r = subprocess.run([sys.executable, "bench.py", "--save-first-T", t1] + SMALL, cwd=ROOT, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    one = _json_line(r.stdout)
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2", "--master-addr",
           "127.0.0.1", "--master-port", str(_free_port()), "bench.py", "--gpus", "2", "--dist-backend", "gloo",
           "--save-first-T", t2] + SMALL
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    two = _json_line(r.stdout)
    assert two["n_gpus"] == 2 and two["scaling"] == "strong"
    assert two["config"]["parallelism"] == "band-partition x2" and one["config"]["parallelism"] == "replicas x1"
    assert two["band_ranges"] == [[0, 27], [27, 55]]
    assert two["gpu_launches"] == 3 * 2 * 15     # sweep, cell solve, fix-up per inner iteration
    for d in (one, two):
        assert d["value"] > 0 and d["unit"] == "updates/s" and d["roofline"]["bound"] == "hbm"
        assert len(d["roofline"]["sweep_ms_last_step"]) == 15 and d["roofline"]["launch_ms"] > 0
    # the config object is the same in both arms of a run (the reference arm prints it too)
    assert set(one["config"]) == set(two["config"])
    Ta, Tb = np.load(t1), np.load(t2)
    assert np.max(np.abs(Ta - Tb) / Ta) <= 1e-12
