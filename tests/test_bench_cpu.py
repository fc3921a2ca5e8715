"""Host logic of bench.py that needs no GPU: the DRAM-traffic record is used
only while its source key matches the sweep kernels' sources (a kernel
changed since the ncu capture reports no traffic), the committed record's
figures are self-consistent, and the HBM roofline arithmetic."""
import hashlib
import json
import os

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _key(paths):
    h = hashlib.sha256()
    for p in paths:
        h.update(open(p, "rb").read())
    return h.hexdigest()[:16]


def test_traffic_record_needs_the_matching_source_key(tmp_path, monkeypatch):
    src = tmp_path / "kernel.cuh"
    src.write_text("// a sweep kernel\n")
    rec = {"kernel_source_sha": _key([str(src)]), "dram_bytes_per_update": 25.5}
    rec_file = tmp_path / "traffic.json"
    rec_file.write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "KERNEL_SRCS", [str(src)])
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(rec_file))
    assert bench.traffic_per_update() == 25.5
    src.write_text("// a sweep kernel, edited after the capture\n")
    assert bench.traffic_per_update() is None
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(tmp_path / "missing.json"))
    assert bench.traffic_per_update() is None


def test_committed_traffic_record_is_consistent():
    rec = json.load(open(os.path.join(ROOT, "profiles", "sweep_traffic.json")))
    per_update = (rec["dram_bytes_read_per_launch"] + rec["dram_bytes_write_per_launch"]) / rec["updates_per_launch_captured"]
    assert abs(per_update - rec["dram_bytes_per_update"]) <= 1e-3
    # at least the algorithmic 24 bytes (B and I^k read, I^{k+1} written), and not
    # far above them (re-reads would show here first)
    assert bench.BYTES_PER_UPDATE_FP64 <= rec["dram_bytes_per_update"] <= 1.2 * bench.BYTES_PER_UPDATE_FP64
    assert len(rec["kernel_source_sha"]) == 16
    assert all(os.path.exists(p) for p in bench.KERNEL_SRCS)


def test_hbm_roofline_arithmetic():
    r = bench.hbm_roof(2.0e11, 24, {"hbm_gbs": 6000.0})
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert abs(r["achieved"] - 4800.0) < 1e-9 and abs(r["frac"] - 0.8) < 1e-12
