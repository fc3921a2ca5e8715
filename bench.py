"""Throughput benchmark of the phonon-BTE hot path (cell*direction*band updates/s).

Workload (default): 2-D 128x128 cells, 400 directions (20 polar x 20 azimuthal),
55 band-polarisations, FP64 intensities, hot-spot wall, implicit Euler with 15
point-Jacobi inner iterations per time step.  One benchmark step is one time
step: 15 inner iterations, each the fused sweep (upwind fluxes, wall ghosts,
relaxation), per-cell reduction, T_p solve and I0 refresh.

Arms:
  (default)          the CUDA library, inputs resident in HBM, CUDA-event timing.
  --impl reference   the plain FP64 CPU oracle on this machine's host cores, on a
                     bounded sub-grid sample of the same workload.

Beside the metric the JSON line carries: the roofline of the dominant sweep
kernel (FP64 pipe, with its HBM figures and the ncu DRAM traffic of the
committed record), the end-to-end rate through the C ABI with host buffers,
SM clocks sampled during the timed region, the launch count, the oracle's own
rate on the host cores (all cores on the full grid, and one thread on a 32x32
sub-grid), "accuracy" (max |dT_L| of the first, untimed step against the FP64
oracle's run of the same step on the full grid) and the reduced-precision,
batched, paper-device, sweep-ordered and unstructured variants.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
For N > 1 launch with torch.distributed.run; every rank runs one replica of the
workload on its own GPU (the path has no exchange step between replicas).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "cell·dir·band updates/s and % HBM roofline at stated max|ΔT| vs FP64 oracle"
UNIT = "updates/s"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "sweep_traffic.json")
KERNEL_SRCS = [os.path.join(ROOT, "paper_2305_19400_gb300", "csrc", f) for f in ("bte_sweep.cuh", "bte_store.cuh")]
# FP64 pipe peak: the nominal 1.25 TFLOP/s corresponds to 2 DFMA/clk/SM on 152 SMs at 2070 MHz.
FP64_PEAK_FLOPS = 2 * 2 * 152 * 2.070e9
# Algorithmic work of one 2-D implicit update: A_n*I^n + A_x*I_x + A_y*I_y + A_s*I0 (4 mul + 3 add)
# and the reduction G_b += w_d*I (1 mul + 1 add); bytes: I^n read, I^k read once, I^{k+1} written.
# A_n*I^n is the same in every inner iteration of a step: computed (and kept) in the first,
# so the later ones take 1 mul fewer.
FLOPS_PER_UPDATE_2D = 9
FLOPS_PER_UPDATE_2D_LATER = 8
BYTES_PER_UPDATE_FP64 = 24


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--nx", type=int, default=128)
    ap.add_argument("--ny", type=int, default=128)
    ap.add_argument("--ninner", type=int, default=15)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--oracle-only", action="store_true", help=argparse.SUPPRESS)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-tune", action="store_true", help="plain launches: no autotuning, no CUDA graph")
    ap.add_argument("--band-partition", action="store_true",
                    help="with N > 1 ranks: split the bands of the one workload over the ranks (Sec. 3.3) and sum the "
                         "per-cell energy partials with an NCCL all-reduce each inner iteration (strong scaling), "
                         "instead of N independent replicas")
    return ap.parse_args()


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


class ClockSampler:
    """nvidia-smi clock/throttle samples every 200 ms while running."""

    FIELDS = ["index", "clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.active",
              "clocks_event_reasons.hw_slowdown", "clocks_event_reasons.hw_thermal_slowdown",
              "clocks_event_reasons.sw_thermal_slowdown", "clocks_event_reasons.sw_power_cap"]

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + ",".join(self.FIELDS), "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=5)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def read_peaks():
    try:
        return json.load(open(PEAKS_FILE)), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def traffic_per_update():
    """DRAM bytes per update of the sweep from the committed ncu summary, or None
    when the kernel source changed since the counters were taken."""
    try:
        rec = json.load(open(TRAFFIC_FILE))
    except (OSError, ValueError):
        return None
    hsh = hashlib.sha256()
    for f in KERNEL_SRCS:
        hsh.update(open(f, "rb").read())
    sha = hsh.hexdigest()[:16]
    if rec.get("kernel_source_sha") != sha:
        return None
    return rec.get("dram_bytes_per_update")


# ----------------------------------------------------------------------------- reference arm
def reference_sample(nx_sub=16, ny_sub=16):
    from paper_2305_19400_gb300 import workloads as W
    wl = W.cfg2(nx_sub, ny_sub, nsteps=1, ninner=15)
    return wl


def run_oracle_sample(wl):
    """One time step (15 inner iterations) of the oracle on the sample; returns (updates, seconds)."""
    from oracle import oracle as O
    g = wl.geoms[0]
    p = O.Problem(g, O.dirs_for(wl.dirs), wl.bands)
    st = p.init_state(g.T_init)
    t0 = time.perf_counter()
    p.run(st, wl.dt, wl.nsteps, wl.ninner)
    return wl.updates, time.perf_counter() - t0, st


def run_oracle_only(args):
    """One oracle time step on an nx x ny sub-grid of the workload, printed as JSON; run in a
    child process so that OMP_NUM_THREADS set for it takes effect."""
    from oracle import oracle as O
    from paper_2305_19400_gb300 import workloads as W
    O.build()
    wl = W.cfg2(args.nx, args.ny, nsteps=1, ninner=args.ninner)
    u, s, _ = run_oracle_sample(wl)
    print(json.dumps({"updates": u, "seconds": s, "cores": O.num_threads()}), flush=True)
    return 0


def oracle_single_thread(ninner, n=32):
    """The oracle with one OpenMP thread on an n x n sub-grid (same directions, bands and walls)."""
    import subprocess
    env = dict(os.environ, OMP_NUM_THREADS="1")
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-only", "--nx", str(n), "--ny", str(n),
                        "--ninner", str(ninner)], env=env, capture_output=True, text=True, check=True)
    rec = json.loads(r.stdout.strip().splitlines()[-1])
    return {"value": rec["updates"] / rec["seconds"], "unit": UNIT, "cores": rec["cores"],
            "sample": f"{n}x{n} sub-grid, 1 time step x {ninner} inner iterations "
                      f"({rec['updates']:.3g} updates, {rec['seconds']:.1f} s)"}


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    from oracle import oracle as O
    O.build()
    wl = reference_sample()
    for _ in range(args.warmup):
        run_oracle_sample(wl)
    tot_u, tot_s = 0, 0.0
    for _ in range(args.steps):
        u, s, _ = run_oracle_sample(wl)
        tot_u += u
        tot_s += s
    v = tot_u / tot_s
    cores = O.num_threads()
    sample = (f"{wl.geoms[0].nx}x{wl.geoms[0].ny} sub-grid of the 128x128 workload (same directions, bands, walls), "
              f"1 time step x {wl.ninner} inner iterations per benchmark step")
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": 1e3 * tot_s / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": "2d_128x128_400dir_55band_fp64", "sample": sample},
           "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
           "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)
    return 0


# ----------------------------------------------------------------------------- our arm
def cpu_baseline_for(args):
    """The oracle as it stands on this host's cores: the full grid for one time step
    (15 inner iterations), about 10-30 s of CPU work."""
    from oracle import oracle as O
    from paper_2305_19400_gb300 import workloads as W
    O.build()
    wl = W.cfg2(args.nx, args.ny, nsteps=1, ninner=args.ninner)
    u, s, st = run_oracle_sample(wl)
    single = oracle_single_thread(args.ninner)
    # the paper's own device (the FP64 variant of the same name): 20 of its 100 steps
    pd = W.paper_hot_spot(nsteps=20)
    g = pd.geoms[0]
    p = O.Problem(g, O.dirs_for(pd.dirs), pd.bands)
    pst = p.init_state(g.T_init)
    t0 = time.perf_counter()
    p.run(pst, pd.dt, pd.nsteps, pd.ninner)
    sp = time.perf_counter() - t0
    return st, {"value": u / s, "unit": UNIT, "cores": O.num_threads(), "kind": "oracle", "single_thread": single,
                "sample": f"full {args.nx}x{args.ny} grid, 1 time step x {args.ninner} inner iterations ({u:.3g} updates, {s:.1f} s)",
                "paper_device": {"value": pd.dof * pd.nsteps / sp, "unit": UNIT, "ms_per_step": 1e3 * sp / pd.nsteps,
                                 "sample": f"120x120 x 20 x 55, 20 of the 100 steps of 1 ns, one inner iteration each ({sp:.1f} s)"}}


def run_variants(peaks):
    """The reduced-precision, learned and batched forms of the path, each on its own
    workload: FP32 and BF16 storage on the 3-D 64^3 x 400 x 55 workload (15 inner
    iterations per step), FP32 with the learned guess on the 3-D 100x100x50 workload
    (networks trained on the GPU on 1e6 pairs over [250, 400] K before timing; 15 inner
    iterations), the 48-geometry FP32 batch (12 inner iterations) and the paper's own
    device in FP64 (120x120 x 20 in-plane directions x 55, 100 steps of 1 ns, one
    inner iteration each), all with CUDA graphs and the autotuner.  Device-timed like
    the main line; bytes per update are the algorithmic 3 x storage size."""
    import torch
    from paper_2305_19400_gb300 import bte, workloads as W
    out = []
    cases = [("fp32_3d_64^3", lambda: W.cfg3(64), bte.BTE_FP32, 4, 15, False),
             ("bf16_3d_64^3", lambda: W.cfg3(64, "bf16"), bte.BTE_BF16, 4, 15, False),
             ("fp32_learned_3d_100x100x50", lambda: W.cfg4(), bte.BTE_FP32, 3, 15, True),
             ("fp32_batch_48_geometries", lambda: W.cfg5(), bte.BTE_FP32, 3, 12, False),
             ("fp64_paper_device_120x120_20dir", lambda: W.paper_hot_spot(), bte.BTE_FP64, 100, 1, False)]
    for name, mk, prec, steps, ninner, learned in cases:
        wl = mk()
        s = bte.Solver(wl, precision=prec, use_graph=True, learned=learned)
        extra = {}
        if learned:
            t0 = time.perf_counter()
            loss = bte.bte_train_mlp(s.h, 1_000_000, 250.0, 400.0, 4, seed=1)
            extra["mlp_training"] = {"pairs": 1_000_000, "epochs": 4, "loss_A": float(loss[0]),
                                     "loss_B": float(loss[1]), "s": time.perf_counter() - t0}
        choice = bte.bte_autotune(s.h, wl.dt).strip().splitlines()[-1]
        s.step(nsteps=1, ninner=ninner, want_stats=False)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        s.step(nsteps=steps, ninner=ninner, want_stats=False)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        ups = wl.dof * ninner * steps / (ms * 1e-3)
        bpu = {bte.BTE_FP64: 24, bte.BTE_FP32: 12, bte.BTE_BF16: 6}[prec]
        gbs = ups * bpu / 1e9
        hbm = {"bound": "hbm", "achieved": gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
               "frac": gbs / peaks["hbm_gbs"], "bytes_per_update": bpu}
        if prec == bte.BTE_FP64:  # FP64-pipe bound; 9 flop per update without the B reuse (one inner iteration)
            fl = ups * (FLOPS_PER_UPDATE_2D if ninner == 1 else
                        (FLOPS_PER_UPDATE_2D + (ninner - 1) * FLOPS_PER_UPDATE_2D_LATER) / ninner)
            roof = {"bound": "alu", "achieved": fl / 1e12, "peak": FP64_PEAK_FLOPS / 1e12, "unit": "TFLOP/s",
                    "frac": fl / FP64_PEAK_FLOPS, "hbm": hbm}
        else:
            roof = hbm
        dtype = {bte.BTE_FP64: "f64", bte.BTE_FP32: "f32", bte.BTE_BF16: "bf16-storage/f32"}[prec]
        out.append({"workload": name, "dtype": dtype, "value": ups,
                    "unit": UNIT, "ms_per_step": ms / steps, "steps": steps, "inner_iterations_per_step": ninner,
                    "cells": sum(g.ncells for g in wl.geoms), "roofline": roof, "launch": choice, **extra})
        if learned:
            st = s.step(nsteps=1, ninner=ninner)[1]
            out[-1]["solves_per_step"] = {k: st[k] for k in ("solves", "solve_evals", "fallbacks")}
        s.close()
        del s
        torch.cuda.empty_cache()
    return out


def run_gs_variant(peaks):
    """Sweep-ordered (Gauss-Seidel) against point-Jacobi inner iterations on the
    128x128 x 400 x 55 FP64 workload with dt = 10 ps (transport CFL up to 7.7,
    where the inner iterations converge slowly).  Per scheme: the device time of
    one inner iteration (3 steps x 15 inner iterations, CUDA graph, autotuned),
    the T_L error of one step after m inner iterations against a 60-iteration
    sweep-ordered step, and from both the time of a step that reaches a
    tolerance."""
    import numpy as np
    import torch
    from paper_2305_19400_gb300 import bte, workloads as W
    dt = 1e-11
    wl = W.cfg2()
    g = wl.geoms[0]
    GS, JAC = bte.BTE_IMPLICIT_GS, bte.BTE_IMPLICIT_JACOBI
    ref = bte.Solver(wl)
    ref.step(nsteps=1, ninner=60, dt=dt, scheme=GS, want_stats=False)
    T_ref = ref.T(0, bte.BTE_T_LATTICE)
    ref.close()
    del ref
    ms_list = (2, 4, 6, 8, 10, 12, 16, 20, 25, 30, 35, 40, 50)
    res = {}
    for name, sch in (("sweep_ordered", GS), ("jacobi", JAC)):
        s = bte.Solver(wl, use_graph=True, autotune=True)
        s.step(nsteps=1, ninner=15, dt=dt, scheme=sch, want_stats=False)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        s.step(nsteps=3, ninner=15, dt=dt, scheme=sch, want_stats=False)
        e1.record()
        torch.cuda.synchronize()
        ms_inner = e0.elapsed_time(e1) / 45
        errs = {}
        for m in ms_list:
            bte.bte_set_initial(s.h, 0, None, g.T_init)
            s.step(nsteps=1, ninner=m, dt=dt, scheme=sch, want_stats=False)
            errs[m] = float(np.max(np.abs(s.T(0, bte.BTE_T_LATTICE) - T_ref)))
        res[name] = {"ms_per_inner_iteration": ms_inner, "updates_per_s": wl.dof / (ms_inner * 1e-3),
                     "max_abs_dTL_K_after_m": errs}
        s.close()
        del s
        torch.cuda.empty_cache()
    for tol in (1e-4, 1e-6):
        for name in res:
            m = next((m for m in ms_list if res[name]["max_abs_dTL_K_after_m"][m] <= tol), None)
            res[name][f"inner_iterations_to_{tol:g}K"] = m
            res[name][f"ms_per_step_to_{tol:g}K"] = None if m is None else m * res[name]["ms_per_inner_iteration"]
    gs = res["sweep_ordered"]
    fl = gs["updates_per_s"] * FLOPS_PER_UPDATE_2D_LATER
    return {"workload": "fp64_sweep_ordered_vs_jacobi_2d_128x128_dt10ps", "dtype": "f64", "value": gs["updates_per_s"],
            "unit": UNIT, "dt_s": dt, "schemes": res,
            "roofline": {"bound": "alu", "achieved": fl / 1e12, "peak": FP64_PEAK_FLOPS / 1e12, "unit": "TFLOP/s",
                         "frac": fl / FP64_PEAK_FLOPS}}


def run_umesh_variant(peaks, precision=None):
    """Unstructured mesh: a 1.28 um square of 128x128 grid squares split into
    32768 jittered triangles, 400 directions (20 x 20) x 55 band-pols, FP64,
    walls hot 305 K / cold 300 K / mirror / diffuse, 15 inner iterations per
    step, device-timed like the main line.  Flops per update: the B-form update
    (2 FMAs) plus one FMA per inflow face and the reduction's FMA, the inflow
    count averaged over the mesh's (cell, direction) pairs."""
    import numpy as np
    import torch
    from paper_2305_19400_gb300 import bte, mesh as M, workloads as W
    m = M.tri_grid(128, 128, 1280e-9, 1280e-9, jitter=0.25, seed=7)
    dirs = W.Dirs("polar_azim", n_polar=20, n_azim=20)
    bands = W.make_bands(40, 15, 19406)
    bc = {0: (bte.BTE_BC_ISOTHERMAL, 305.0), 1: (bte.BTE_BC_ISOTHERMAL, 300.0),
          2: (bte.BTE_BC_SPECULAR, None), 3: (bte.BTE_BC_DIFFUSE, None)}
    prec = bte.BTE_FP64 if precision is None else precision
    s = bte.UMeshSolver(m, dirs, bands, bc, precision=prec)
    dt, ninner, steps = 1e-12, 15, 3
    s.step(dt, 1, ninner, want_stats=False)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    s.step(dt, steps, ninner, want_stats=False)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    dof = m.ncells * dirs.nd * len(bands.vg)
    ups = dof * ninner * steps / (ms * 1e-3)
    # inflow faces per (cell, direction): the in-plane part of S_d points along the azimuth
    phi = (np.arange(dirs.n_azim) + 0.5) * 2 * np.pi / dirs.n_azim
    sdir = np.stack([np.cos(phi), np.sin(phi)], axis=1)
    sn = m.nA[:, :2] @ sdir.T                       # [face, azimuth], out of the owner
    inflow = (sn < 0).sum() + (sn[m.neighbor >= 0] > 0).sum()
    nin = inflow / (m.ncells * dirs.n_azim)
    flops = 2.0 * (2 + nin) + 2.0
    fl = ups * flops
    s.close()
    del s
    torch.cuda.empty_cache()
    if prec == bte.BTE_FP64:
        roof = {"bound": "alu", "achieved": fl / 1e12, "peak": FP64_PEAK_FLOPS / 1e12, "unit": "TFLOP/s",
                "frac": fl / FP64_PEAK_FLOPS, "flop_per_update": flops}
    else:  # B (or I^n), R and I^{k+1} in the sweep, I^{k+1} again in the per-cell step
        bpu = 16 if prec == bte.BTE_FP32 else 10   # BF16: 2-byte I, R stays a 4-byte float
        gbs = ups * bpu / 1e9
        roof = {"bound": "hbm", "achieved": gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": gbs / peaks["hbm_gbs"], "bytes_per_update": bpu}
    name = {bte.BTE_FP64: "fp64", bte.BTE_FP32: "fp32", bte.BTE_BF16: "bf16"}[prec]
    return {"workload": f"{name}_unstructured_32768_triangles_400dir",
            "dtype": {bte.BTE_FP64: "f64", bte.BTE_FP32: "f32", bte.BTE_BF16: "bf16-storage/f32"}[prec],
            "value": ups, "unit": UNIT,
            "ms_per_step": ms / steps, "steps": steps, "inner_iterations_per_step": ninner, "cells": m.ncells,
            "inflow_faces_per_cell_direction": float(nin), "roofline": roof}


def main():
    args = parse()
    if args.oracle_only:
        return run_oracle_only(args)
    if args.impl == "reference":
        return run_reference(args)
    world, rank, local = dist_env()
    import numpy as np
    import torch

    from paper_2305_19400_gb300 import build as B, bte, workloads as W

    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0:
        B.build()
    if world > 1:
        dist.barrier()
    stream = torch.cuda.current_stream()
    wl = W.cfg2(args.nx, args.ny, nsteps=1, ninner=args.ninner)
    g = wl.geoms[0]
    tuned = not args.no_tune
    partitioned = world > 1 and args.band_partition
    if partitioned:  # contiguous, balanced band ranges; the exchange is an NCCL all-reduce on this stream
        nb = wl.bands.nb
        lo, hi = rank * nb // world, (rank + 1) * nb // world
        solver = bte.Solver(wl, stream=stream, band_range=(lo, hi), exchange=bte.allreduce_exchange())
        own_dof = wl.dof // nb * (hi - lo)
    else:
        solver = bte.Solver(wl, stream=stream, use_graph=tuned)
        own_dof = wl.dof
    tune_choice = bte.bte_autotune(solver.h, wl.dt).strip().splitlines()[-1] if tuned else "untuned"
    updates_per_step = own_dof * args.ninner

    def step():
        rc, st = bte.bte_step(solver.h, wl.dt, 1, args.ninner, bte.BTE_IMPLICIT_JACOBI, want_stats=False)
        return rc

    step()   # the first warm-up step, from the initial state: kept for the accuracy check against the oracle
    TL_first = solver.T(0, bte.BTE_T_LATTICE) if world == 1 else None
    for _ in range(args.warmup - 1):
        step()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ms = e0.elapsed_time(e1)
    clk = clocks.stop()
    t = torch.tensor([ms], dtype=torch.float64, device="cuda")
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max = float(t.item())
    # sweep + fix-up kernel per inner iteration (+ the cell solve after the exchange of a band range)
    launches = (3 if partitioned else 2) * args.steps * args.ninner
    total_updates_per_step = wl.dof * args.ninner if partitioned else world * updates_per_step
    value = total_updates_per_step * args.steps / (ms_max * 1e-3)

    # sanity: the state is finite and physical after the timed run
    TL = solver.T(0, bte.BTE_T_LATTICE)
    assert np.all(np.isfinite(TL)) and TL.min() > 299.0 and TL.max() < 311.0, (TL.min(), TL.max())

    # ---- end to end through the C ABI with host buffers: per step, the hot-wall
    # temperatures go host->device (bte_set_bc), one time step runs, and the
    # lattice temperatures come back device->host (bte_get_T).
    e2e = None
    if not args.no_e2e:
        Tw = torch.from_numpy(W.hot_spot_profile(g.ny, 300.0, 10.0, 8.0)).pin_memory()
        Tout = torch.empty(g.ncells, dtype=torch.float64).pin_memory()
        import ctypes as C
        L = bte.lib()
        twp = C.cast(C.c_void_p(Tw.data_ptr()), C.POINTER(C.c_double))
        k_e2e = max(3, min(args.steps, 20))
        for _ in range(2):
            L.bte_set_bc(solver.h, 0, 0, bte.BTE_BC_ISOTHERMAL, twp, 300.0)
            step()
            L.bte_get_T(solver.h, 0, bte.BTE_T_LATTICE, C.c_void_p(Tout.data_ptr()), 0)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(k_e2e):
            rc = L.bte_set_bc(solver.h, 0, 0, bte.BTE_BC_ISOTHERMAL, twp, 300.0)
            assert rc == 0, bte.bte_last_error(solver.h)
            step()
            rc = L.bte_get_T(solver.h, 0, bte.BTE_T_LATTICE, C.c_void_p(Tout.data_ptr()), 0)
            assert rc == 0, bte.bte_last_error(solver.h)
        dt_e2e = time.perf_counter() - t0
        te = torch.tensor([dt_e2e], dtype=torch.float64, device="cuda")
        if world > 1:
            dist.all_reduce(te, op=dist.ReduceOp.MAX)
        e2e = {"value": total_updates_per_step * k_e2e / float(te.item()), "unit": UNIT,
               "h2d_bytes_per_step": Tw.numel() * 8, "d2h_bytes_per_step": Tout.numel() * 8, "steps": k_e2e}
    solver.close()

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return 0
    peaks, peak_src = read_peaks()
    # the whole step time (sweeps and fix-ups) charged to the sweeps: a lower bound of the sweep's own rate
    launch_s = ms_max * 1e-3 / (args.steps * args.ninner)
    upd_launch = updates_per_step / args.ninner
    fpu = (FLOPS_PER_UPDATE_2D + (args.ninner - 1) * FLOPS_PER_UPDATE_2D_LATER) / args.ninner
    flops = fpu * upd_launch / launch_s
    hbm = BYTES_PER_UPDATE_FP64 * upd_launch / launch_s / 1e9
    tpu = traffic_per_update()
    roofline = {"bound": "alu", "achieved": flops / 1e12, "peak": FP64_PEAK_FLOPS / 1e12, "unit": "TFLOP/s",
                "frac": flops / FP64_PEAK_FLOPS,
                "traffic": (tpu * upd_launch) if tpu else None,
                "kernel": "sweep_kernel<2, double, MINB, 2> (inner iterations 2..15; iteration 1 is BM=1)",
                "peak_source": "FP64 pipe: 2 DFMA/clk/SM x 152 SMs x 2070 MHz (nominal 1.25 TFLOP/s)",
                "flops": ("method flops per update: 9 in inner iteration 1, 8 in the later ones; they include "
                          "the reduction's multiply and add, which this kernel runs exactly in fixed point on the "
                          "integer pipe, so the fraction of the FP64 pipe's peak can slightly exceed 1"),
                "hbm": {"achieved": hbm, "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": hbm / peaks["hbm_gbs"],
                        "peak_source": f"hbm_gbs of {peak_src} peaks"}}
    cpu = accuracy = None
    if world == 1 and not args.no_cpu_baseline:
        ost, cpu = cpu_baseline_for(args)
        accuracy = {"max_abs_dTL_K": float(np.max(np.abs(TL_first - ost["TL"]))),
                    "max_rel_dTL": float(np.max(np.abs(TL_first - ost["TL"]) / ost["TL"])),
                    "against": f"FP64 oracle, full {args.nx}x{args.ny} grid, first time step x {args.ninner} "
                               "inner iterations, same launch configuration as the timed steps"}
        del ost
    variants = None
    if world == 1 and not args.no_variants:
        variants = run_variants(peaks)
        variants.append(run_gs_variant(peaks))
        variants.append(run_umesh_variant(peaks))
        variants.append(run_umesh_variant(peaks, 1))
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
           "scaling": "strong" if partitioned else "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": f"2d_{args.nx}x{args.ny}_400dir_55band_fp64", "cells": g.ncells, "directions": 400,
                      "band_pols": 55, "inner_iterations_per_step": args.ninner, "dt_s": wl.dt,
                      "scheme": "implicit Euler, point-Jacobi inner iterations",
                      "l2": "inputs larger than L2 (three FP64 intensity buffers of %.2f GB each)" % (wl.dof * 8 / 1e9),
                      "launch": ("CUDA graph per time step, autotuned (cells_per_cta,threads,grid,min_ctas_variant): "
                                 + tune_choice) if tuned else "eager launches, default tiles",
                      "parallelism": f"band-partition x{world}" if partitioned else f"replicas x{world}"},
           "gpu_launches": launches, "clocks": clk, "roofline": roofline, "e2e": e2e, "cpu_baseline": cpu,
           "accuracy": accuracy, "variants": variants}
    print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
