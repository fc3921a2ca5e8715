"""Throughput benchmark of the phonon-BTE hot path (cell*direction*band updates/s).

Workload (default): 2-D 128x128 cells, 400 directions (20 polar x 20 azimuthal),
55 band-polarisations, FP64 intensities, hot-spot wall, implicit Euler with 15
point-Jacobi inner iterations per time step.  One benchmark step is one time
step: 15 inner iterations, each the fused sweep (upwind fluxes, wall ghosts,
relaxation), per-cell reduction, T_p solve and I0 refresh.  FP64 storage; the
sweep's update runs in double-float arithmetic on the FP32 pipe (the default
of the library's FP64 mode; a variant times the strict IEEE-FP64 form).

Arms:
  (default)          the CUDA library, inputs resident in HBM, CUDA-event timing.
  --impl reference   the plain FP64 CPU oracle on this machine's host cores, on a
                     bounded sub-grid sample of the same workload (the sample the
                     CPU-baseline leg of the default arm also times).

Beside the metric the JSON line carries: the roofline of the dominant sweep
kernel (HBM bytes over its per-launch time, measured by CUDA events recorded
around each sweep inside the timed steps, against the measured copy
bandwidth; the FP32-pipe load of its double-float arithmetic against the
library's measured FMA peak; and the ncu DRAM traffic of the committed
record), the end-to-end rate through the C ABI with host buffers, SM clocks
sampled during the timed region, the launch count, the oracle's own rate on
the host cores, "accuracy" (max |dT_L| of the first, untimed step against
the FP64 oracle's run of the same step on the full grid) and the
reduced-precision, learned (with and without the network), batched,
strict-FP64, paper-device (100 steps, and its full 20 us run with an energy
record), sweep-ordered and unstructured variants.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
For N > 1 launch with torch.distributed.run: the ranks split the bands of the
one workload (Sec. 3.3 band partition; contiguous balanced ranges) and sum the
per-cell energy partials with an all-reduce every inner iteration (NCCL on the
solver's stream; --dist-backend gloo reduces a host copy).  --replicas runs N
independent copies of the workload instead.
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
KERNEL_SRCS = [os.path.join(ROOT, "paper_2305_19400_gb300", "csrc", f) for f in ("bte_sweep_ff.cuh", "bte_ff.cuh", "bte_sweep.cuh", "bte_store.cuh")]
# Algorithmic bytes of one implicit update: I^n (or B) read, I^k read once, I^{k+1} written.
BYTES_PER_UPDATE_FP64 = 24
# Work of the dominant kernel (the double-float sweep of inner iterations 2..n-1,
# 2-D): per lane step of two bands, 3 products of 4 packed ops (c_x u_x, c_y u_y,
# and R times the sum), 3 pair sums of 8 (the two products, the source term,
# B), a normalisation of 3 and the direction sum's accumulation of 8 = 47
# packed f32x2 instructions for 2 updates, i.e. 47 FP32 lane operations per
# update; counted against the measured packed-FMA rate in lane operations.
FP32_LANE_OPS_PER_UPDATE_FF_2D = 47
# The strict IEEE-FP64 sweep: 3 FMAs per update (B + A_x I_x + A_y I_y + A_s I0)
# in inner iterations 2..n, 4 in the first (A_n I^n).
FP64_FMAS_PER_UPDATE_2D = 3


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
    ap.add_argument("--replicas", action="store_true",
                    help="with N > 1 ranks: N independent copies of the workload (weak scaling) instead of the band "
                         "partition of the one workload")
    ap.add_argument("--dist-backend", default="nccl", choices=["nccl", "gloo"],
                    help="process group of N > 1 ranks (gloo: the exchange reduces a host copy)")
    ap.add_argument("--save-first-T", default=None, help=argparse.SUPPRESS)   # rank 0: T_L after the first step (.npy)
    return ap.parse_args()


# The CPU sample of the workload that the reference arm and the CPU-baseline leg
# both time: a 64x64 sub-grid (same directions, bands, wall kinds; the hot spot
# scaled to the sub-grid's height), one time step of 15 inner iterations.
SAMPLE_NX, SAMPLE_NY = 64, 64


def workload_config(args, world, partitioned):
    """The JSON "config" object, identical in both arms."""
    from paper_2305_19400_gb300 import workloads as W
    wl = W.cfg2(args.nx, args.ny, nsteps=1, ninner=args.ninner)
    return {"workload": f"2d_{args.nx}x{args.ny}_400dir_55band_fp64", "cells": wl.geoms[0].ncells,
            "directions": 400, "band_pols": 55, "inner_iterations_per_step": args.ninner, "dt_s": wl.dt,
            "scheme": "implicit Euler, point-Jacobi inner iterations",
            "parallelism": (f"band-partition x{world}" if partitioned else f"replicas x{world}")}


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
def run_oracle_sample(wl):
    """One time step (15 inner iterations) of the oracle on the sample; returns (updates, seconds, state)."""
    from oracle import oracle as O
    g = wl.geoms[0]
    p = O.Problem(g, O.dirs_for(wl.dirs), wl.bands)
    st = p.init_state(g.T_init)
    t0 = time.perf_counter()
    p.run(st, wl.dt, wl.nsteps, wl.ninner)
    return wl.updates, time.perf_counter() - t0, st


def sample_workload(ninner):
    from paper_2305_19400_gb300 import workloads as W
    return W.cfg2(SAMPLE_NX, SAMPLE_NY, nsteps=1, ninner=ninner)


def sample_text(ninner):
    return (f"{SAMPLE_NX}x{SAMPLE_NY} sub-grid of the workload (same directions, bands and wall kinds), "
            f"1 time step x {ninner} inner iterations per benchmark step")


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
    env = dict(os.environ, OMP_NUM_THREADS="1")
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-only", "--nx", str(n), "--ny", str(n),
                        "--ninner", str(ninner)], env=env, capture_output=True, text=True, check=True)
    rec = json.loads(r.stdout.strip().splitlines()[-1])
    return {"value": rec["updates"] / rec["seconds"], "unit": UNIT, "cores": rec["cores"],
            "sample": f"{n}x{n} sub-grid, 1 time step x {ninner} inner iterations "
                      f"({rec['updates']:.3g} updates, {rec['seconds']:.1f} s)"}


def run_reference(args):
    """The reference arm: the FP64 oracle as it stands on the host cores, each
    benchmark step one oracle time step on the shared CPU sample."""
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    from oracle import oracle as O
    O.build()
    wl = sample_workload(args.ninner)
    for _ in range(args.warmup):
        run_oracle_sample(wl)
    tot_u, tot_s = 0, 0.0
    for _ in range(args.steps):
        u, s, _ = run_oracle_sample(wl)
        tot_u += u
        tot_s += s
    v = tot_u / tot_s
    cores = O.num_threads()
    sample = sample_text(args.ninner)
    partitioned = world > 1 and not args.replicas
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": 1e3 * tot_s / args.steps, "higher_is_better": True,
           "scaling": "strong" if partitioned else "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": workload_config(args, world, partitioned),
           "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
           "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)
    return 0


# ----------------------------------------------------------------------------- our arm
def cpu_baseline_for(args, paper_TL100=None):
    """The oracle as it stands on this host's cores: the shared CPU sample (the
    reported baseline, as in the reference arm), the full grid for one time step
    (the accuracy pairing of the main line), one thread on a 32x32 sub-grid, and
    the paper's device: its first 100 steps, timed, and compared with the GPU's
    T_L after the same 100 steps."""
    import numpy as np
    from oracle import oracle as O
    from paper_2305_19400_gb300 import workloads as W
    O.build()
    su, ss, _ = run_oracle_sample(sample_workload(args.ninner))
    wl = W.cfg2(args.nx, args.ny, nsteps=1, ninner=args.ninner)
    u, s, st = run_oracle_sample(wl)
    single = oracle_single_thread(args.ninner)
    pd = W.paper_hot_spot(nsteps=100)
    g = pd.geoms[0]
    p = O.Problem(g, O.dirs_for(pd.dirs), pd.bands)
    pst = p.init_state(g.T_init)
    t0 = time.perf_counter()
    p.run(pst, pd.dt, pd.nsteps, pd.ninner)
    sp = time.perf_counter() - t0
    paper = {"value": pd.dof * pd.nsteps / sp, "unit": UNIT, "ms_per_step": 1e3 * sp / pd.nsteps,
             "sample": f"120x120 x 20 x 55, the first 100 steps of 1 ns, one inner iteration each ({sp:.1f} s)"}
    if paper_TL100 is not None:
        paper["gpu_vs_oracle_after_100_steps"] = {
            "max_rel_dTL": float(np.max(np.abs(paper_TL100 - pst["TL"]) / pst["TL"])),
            "max_abs_dTL_K": float(np.max(np.abs(paper_TL100 - pst["TL"])))}
    return st, {"value": su / ss, "unit": UNIT, "cores": O.num_threads(), "kind": "oracle",
                "sample": sample_text(args.ninner) + f" ({su:.3g} updates, {ss:.1f} s)",
                "full_grid": {"value": u / s, "unit": UNIT,
                              "sample": f"full {args.nx}x{args.ny} grid, 1 time step x {args.ninner} inner iterations "
                                        f"({u:.3g} updates, {s:.1f} s)"},
                "single_thread": single, "paper_device": paper}


def timed_steps(s, steps, ninner, **kw):
    """Device time (ms) of `steps` time steps of solver s, CUDA events on the current stream."""
    import torch
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    s.step(nsteps=steps, ninner=ninner, want_stats=False, **kw)
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


def hbm_roof(ups, bpu, peaks):
    gbs = ups * bpu / 1e9
    return {"bound": "hbm", "achieved": gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": gbs / peaks["hbm_gbs"], "bytes_per_update": bpu}


def run_variants(peaks, fp64_peak):
    """The reduced-precision, learned and batched forms of the path, each on its own
    workload: FP32 and BF16 storage on the 3-D 64^3 x 400 x 55 workload (15 inner
    iterations per step), FP32 with and without the learned guess on the 3-D
    100x100x50 workload (networks trained on the GPU on 1e6 pairs over [250, 400] K
    before timing; 15 inner iterations), the 48-geometry FP32 batch (12 inner
    iterations), the main workload with strict IEEE-FP64 arithmetic, and the paper's
    own device in FP64 (120x120 x 20 in-plane directions x 55, 100 steps of 1 ns, one
    inner iteration each), all with CUDA graphs and the autotuner.  Device-timed like
    the main line; bytes per update are the algorithmic 3 x storage size."""
    import torch
    from paper_2305_19400_gb300 import bte, workloads as W
    out = []
    cases = [("fp32_3d_64^3", lambda: W.cfg3(64), bte.BTE_FP32, 4, 15, {}),
             ("bf16_3d_64^3", lambda: W.cfg3(64, "bf16"), bte.BTE_BF16, 4, 15, {}),
             ("fp32_learned_3d_100x100x50", lambda: W.cfg4(), bte.BTE_FP32, 3, 15, {"learned": True}),
             ("fp32_no_network_3d_100x100x50", lambda: W.cfg4(), bte.BTE_FP32, 3, 15, {}),
             ("fp32_batch_48_geometries", lambda: W.cfg5(), bte.BTE_FP32, 3, 12, {}),
             ("fp64_strict_2d_128x128", lambda: W.cfg2(), bte.BTE_FP64, 3, 15, {"fp64_strict": True}),
             ("fp64_paper_device_120x120_20dir", lambda: W.paper_hot_spot(), bte.BTE_FP64, 100, 1, {})]
    for name, mk, prec, steps, ninner, kw in cases:
        wl = mk()
        s = bte.Solver(wl, precision=prec, use_graph=True, **kw)
        extra = {}
        if kw.get("learned"):
            t0 = time.perf_counter()
            loss = bte.bte_train_mlp(s.h, 1_000_000, 250.0, 400.0, 4, seed=1)
            extra["mlp_training"] = {"pairs": 1_000_000, "epochs": 4, "loss_A": float(loss[0]),
                                     "loss_B": float(loss[1]), "s": time.perf_counter() - t0}
        choice = bte.bte_autotune(s.h, wl.dt).strip().splitlines()[-1]
        s.step(nsteps=1, ninner=ninner, want_stats=False)
        ms = timed_steps(s, steps, ninner)
        ups = wl.dof * ninner * steps / (ms * 1e-3)
        bpu = {bte.BTE_FP64: 24, bte.BTE_FP32: 12, bte.BTE_BF16: 6}[prec]
        roof = hbm_roof(ups, bpu, peaks)
        if kw.get("fp64_strict"):  # FP64-pipe bound: FMAs per update against the measured DFMA rate
            fmas = (FP64_FMAS_PER_UPDATE_2D + 1 + (ninner - 1) * FP64_FMAS_PER_UPDATE_2D) / ninner
            fl = 2.0 * fmas * ups
            roof = {"bound": "alu", "achieved": fl / 1e12, "peak": fp64_peak / 1e12, "unit": "TFLOP/s",
                    "frac": fl / fp64_peak, "fmas_per_update": fmas,
                    "peak_source": "bte_measure_peak(BTE_PEAK_FP64_FMA), measured", "hbm": roof}
        dtype = {bte.BTE_FP64: "f64 storage, double-float (f32x2) sweep arithmetic", bte.BTE_FP32: "f32",
                 bte.BTE_BF16: "bf16-storage/f32"}[prec]
        if kw.get("fp64_strict"):
            dtype = "f64"
        out.append({"workload": name, "dtype": dtype, "value": ups,
                    "unit": UNIT, "ms_per_step": ms / steps, "steps": steps, "inner_iterations_per_step": ninner,
                    "cells": sum(g.ncells for g in wl.geoms), "roofline": roof, "launch": choice, **extra})
        if "3d_100x100x50" in name:
            st = s.step(nsteps=1, ninner=ninner)[1]
            out[-1]["solves_per_step"] = {k: st[k] for k in ("solves", "solve_evals", "fallbacks")}
        s.close()
        del s
        torch.cuda.empty_cache()
    learned = next(v for v in out if v["workload"] == "fp32_learned_3d_100x100x50")
    plain = next(v for v in out if v["workload"] == "fp32_no_network_3d_100x100x50")
    learned["gain_over_no_network"] = {
        "value_no_network": plain["value"], "frac": learned["value"] / plain["value"] - 1.0,
        "exact_evaluations_per_step": [learned["solves_per_step"]["solve_evals"],
                                       plain["solves_per_step"]["solve_evals"]],
        "note": "steady operation solves every cell from its cached model; the network only starts the exact "
                "solve of the fix-up cells"}
    return out


def run_paper_device_20us(peaks):
    """The paper's device (Sec. 3.1-3.2) for its full 20 us: 20,000 implicit
    steps of 1 ns (one inner iteration each) from the 300 K start, in chunks of
    10 steps; after each chunk the stored energy sum_P V E_L(P) and the four
    wall powers (the no-allocation wall flux times the wall length, per metre
    of depth) are sampled.  Reports the chunks' device time, the energy record
    (stored-energy change against the time integral of the net wall power,
    trapezoid rule over the samples), the final powers, the T_L range, the
    hot-wall and centre-line profiles, and T_L after the first 100 steps (the
    oracle comparison runs in the CPU-baseline leg)."""
    import numpy as np
    import torch
    from paper_2305_19400_gb300 import bte, workloads as W
    wl = W.paper_hot_spot(nsteps=20000)
    g = wl.geoms[0]
    s = bte.Solver(wl, use_graph=True)
    choice = bte.bte_autotune(s.h, wl.dt).strip().splitlines()[-1]
    vol = g.dx * g.dy
    length = [g.ny * g.dy, g.ny * g.dy, g.nx * g.dx, g.nx * g.dx]

    def sample():
        EL = np.zeros(g.ncells)
        bte.bte_get_T(s.h, 0, bte.BTE_E_LATTICE, EL)
        qw = np.zeros(4)
        bte.bte_get_wall_flux_noalloc(s.h, 0, qw)
        return float(EL.sum() * vol), qw * np.array(length)

    chunk, nchunks = 10, wl.nsteps // 10
    E0, P0 = sample()
    E, P = [E0], [P0]
    dev_ms = 0.0
    TL100 = None
    for c in range(nchunks):
        dev_ms += timed_steps(s, chunk, 1)
        e, p = sample()
        E.append(e)
        P.append(p)
        if (c + 1) * chunk == 100:
            TL100 = s.T(0, bte.BTE_T_LATTICE)
    E = np.array(E)
    P = np.array(P)
    net = P.sum(axis=1)
    dt_chunk = chunk * wl.dt
    inflow = float(np.sum(0.5 * (net[1:] + net[:-1])) * dt_chunk)   # energy that left through the walls
    dE = float(E[-1] - E[0])
    TL = s.T(0, bte.BTE_T_LATTICE).reshape(g.ny, g.nx)
    ups = wl.dof * wl.nsteps / (dev_ms * 1e-3)
    rows = list(range(0, g.ny, 10)) + [g.ny // 2]
    out = {"workload": "fp64_paper_device_120x120_20dir_20us",
           "dtype": "f64 storage, double-float (f32x2) sweep arithmetic", "value": ups, "unit": UNIT,
           "steps": wl.nsteps, "inner_iterations_per_step": 1, "ms_per_step": dev_ms / wl.nsteps,
           "simulated_s": wl.nsteps * wl.dt, "launch": choice, "roofline": hbm_roof(ups, 24, peaks),
           "energy_record": {
               "stored_J_per_m": [float(E[0]), float(E[-1])], "stored_change_J_per_m": dE,
               "net_wall_outflow_integral_J_per_m": inflow,
               "balance_residual_rel": (dE + inflow) / max(abs(dE), abs(inflow), 1e-300),
               "final_wall_power_W_per_m": {"-x (hot)": float(P[-1, 0]), "+x (cold)": float(P[-1, 1]),
                                            "-y": float(P[-1, 2]), "+y": float(P[-1, 3])},
               "final_net_over_hot_wall": float(net[-1] / abs(P[-1, 0])),
               "stored_over_inflow": dE / max(-inflow, 1e-300),
               "samples": int(len(E)), "sample_every_steps": chunk,
               "note": "one point-Jacobi inner iteration per 1 ns step: with beta_b dt up to 1e3 the lagged "
                       "scattering source and upwind values are far from the step's converged backward-Euler "
                       "solution, which alone conserves energy; the FP64 oracle on a 24x24 version of the device "
                       "stores 0.05, 0.39, 0.84, 0.999 and 1.000 of the wall inflow with 1, 16, 64, 256 and 1024 "
                       "inner iterations per step"},
           "TL_K": {"min": float(TL.min()), "max": float(TL.max()), "mean": float(TL.mean())},
           "hot_wall_column_TL_K": {str(j): float(TL[j, 0]) for j in sorted(set(rows))},
           "centre_line_TL_K": {str(i): float(TL[g.ny // 2, i]) for i in range(0, g.nx, 10)}}
    s.close()
    del s
    torch.cuda.empty_cache()
    return out, TL100


def run_gs_variant(peaks, fp64_peak):
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
    fl = gs["updates_per_s"] * 2 * FP64_FMAS_PER_UPDATE_2D   # the pass's B-form update: 3 FMAs
    return {"workload": "fp64_sweep_ordered_vs_jacobi_2d_128x128_dt10ps", "dtype": "f64", "value": gs["updates_per_s"],
            "unit": UNIT, "dt_s": dt, "schemes": res,
            "roofline": {"bound": "alu", "achieved": fl / 1e12, "peak": fp64_peak / 1e12, "unit": "TFLOP/s",
                         "frac": fl / fp64_peak, "peak_source": "bte_measure_peak(BTE_PEAK_FP64_FMA), measured"}}


def run_umesh_variant(peaks, fp64_peak, precision=None):
    """Unstructured mesh: a 1.28 um square of 128x128 grid squares split into
    32768 jittered triangles, 400 directions (20 x 20) x 55 band-pols, FP64,
    walls hot 305 K / cold 300 K / mirror / diffuse, 15 inner iterations per
    step, device-timed like the main line.  FP64 work per update: the B-form
    update (2 FMAs) plus one FMA per inflow face, the inflow count averaged
    over the mesh's (cell, direction) pairs (the per-cell sums of the separate
    reduction run in fixed point on the integer pipe)."""
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
    flops = 2.0 * (2 + nin)
    fl = ups * flops
    s.close()
    del s
    torch.cuda.empty_cache()
    if prec == bte.BTE_FP64:
        roof = {"bound": "alu", "achieved": fl / 1e12, "peak": fp64_peak / 1e12, "unit": "TFLOP/s",
                "frac": fl / fp64_peak, "flop_per_update": flops,
                "peak_source": "bte_measure_peak(BTE_PEAK_FP64_FMA), measured"}
    else:  # algorithmic: I^n (or B), I^k (each row once from DRAM) and I^{k+1}; the sweep also
        # reads the R table and the per-cell step reads I^{k+1} again (not counted)
        bpu = 12 if prec == bte.BTE_FP32 else 6
        gbs = ups * bpu / 1e9
        roof = {"bound": "hbm", "achieved": gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": gbs / peaks["hbm_gbs"], "bytes_per_update": bpu}
    name = {bte.BTE_FP64: "fp64", bte.BTE_FP32: "fp32", bte.BTE_BF16: "bf16"}[prec]
    return {"workload": f"{name}_unstructured_32768_triangles_400dir",
            "dtype": {bte.BTE_FP64: "f64", bte.BTE_FP32: "f32", bte.BTE_BF16: "bf16-storage/f32"}[prec],
            "value": ups, "unit": UNIT,
            "ms_per_step": ms / steps, "steps": steps, "inner_iterations_per_step": ninner, "cells": m.ncells,
            "inflow_faces_per_cell_direction": float(nin), "roofline": roof}


def measure_peaks(local):
    """The library's FMA-loop peaks of this GPU, with the SM clock sampled while they run."""
    from paper_2305_19400_gb300 import bte
    clk = ClockSampler(local)
    clk.start()
    time.sleep(0.3)
    f64, _ = bte.bte_measure_peak(bte.BTE_PEAK_FP64_FMA)
    f32, _ = bte.bte_measure_peak(bte.BTE_PEAK_FP32X2_FMA)
    time.sleep(0.3)
    c = clk.stop()
    return {"fp64_fma_flops": f64, "fp32x2_fma_flops": f32, "sm_mhz": c["sm_mhz"], "reasons": c["reasons"]}


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

    ndev = torch.cuda.device_count()
    dev = local % max(ndev, 1)   # ranks beyond the GPU count share devices (tests on one GPU)
    torch.cuda.set_device(dev)
    if world > 1:
        import torch.distributed as dist
        if args.dist_backend == "nccl":
            dist.init_process_group("nccl", device_id=torch.device("cuda", dev))
        else:
            dist.init_process_group("gloo")
    if rank == 0:
        B.build()
    if world > 1:
        dist.barrier()
    stream = torch.cuda.current_stream()
    wl = W.cfg2(args.nx, args.ny, nsteps=1, ninner=args.ninner)
    g = wl.geoms[0]
    tuned = not args.no_tune
    partitioned = world > 1 and not args.replicas
    if partitioned:  # contiguous, balanced band ranges; the exchange is an all-reduce on this stream
        nb = wl.bands.nb
        lo, hi = rank * nb // world, (rank + 1) * nb // world
        solver = bte.Solver(wl, stream=stream, band_range=(lo, hi), exchange=bte.allreduce_exchange())
        own_dof = wl.dof // nb * (hi - lo)
    else:
        solver = bte.Solver(wl, stream=stream, use_graph=tuned)
        own_dof = wl.dof
    tune_choice = bte.bte_autotune(solver.h, wl.dt).strip().splitlines()[-1] if tuned else "untuned"
    updates_per_step = own_dof * args.ninner
    peaks_lib = measure_peaks(dev) if rank == 0 else None
    bte.bte_set_sweep_timing(solver.h, True)   # events around each sweep, recorded inside the step (graph)

    def step():
        rc, st = bte.bte_step(solver.h, wl.dt, 1, args.ninner, bte.BTE_IMPLICIT_JACOBI, want_stats=False)
        return rc

    step()   # the first warm-up step, from the initial state: kept for the accuracy check against the oracle
    TL_first = solver.T(0, bte.BTE_T_LATTICE)
    if args.save_first_T and rank == 0:
        np.save(args.save_first_T, TL_first)
    for _ in range(args.warmup - 1):
        step()
    torch.cuda.synchronize()
    clocks = ClockSampler(dev)
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
    sweep_ms = bte.bte_sweep_times(solver.h)   # the sweeps of the last timed step, in inner-iteration order
    red_dev = "cuda" if args.dist_backend == "nccl" else "cpu"   # where the timing all-reduces run
    t = torch.tensor([ms], dtype=torch.float64, device=red_dev)
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
        te = torch.tensor([dt_e2e], dtype=torch.float64, device=red_dev)
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
    # roofline of the dominant kernel: the middle inner iterations' sweep (the
    # double-float variant that reads and writes ff iterates), per launch
    mid = sweep_ms[1:-1] if len(sweep_ms) > 2 else sweep_ms
    launch_ms = float(np.mean(mid))
    upd_launch = updates_per_step / args.ninner
    hbm = BYTES_PER_UPDATE_FP64 * upd_launch / (launch_ms * 1e-3) / 1e9
    tpu = traffic_per_update()
    lane_ops = FP32_LANE_OPS_PER_UPDATE_FF_2D * upd_launch / (launch_ms * 1e-3)
    lane_peak = peaks_lib["fp32x2_fma_flops"] / 2.0      # lane FMAs per second
    roofline = {"bound": "hbm", "achieved": hbm, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": hbm / peaks["hbm_gbs"], "traffic": (tpu * upd_launch) if tpu else None,
                "peak_source": f"hbm_gbs of {peak_src} peaks (copy bandwidth)",
                "kernel": "sweep_ff_kernel<2, MINB, 2, 3> (double-float sweep of inner iterations 2..15: "
                          "B and I^k read as ff pairs, I^{k+1} written as ff pairs)",
                "launch_ms": launch_ms, "launches_averaged": len(mid), "bytes_per_update": BYTES_PER_UPDATE_FP64,
                "sweep_ms_last_step": [round(float(x), 4) for x in sweep_ms],
                "timing": "CUDA events recorded by the step graph around each sweep launch, last timed step",
                "step_time_frac_in_sweeps": float(np.sum(sweep_ms) / (ms_max / args.steps)),
                "fp32_pipe": {"achieved_lane_ops": lane_ops, "peak_lane_fmas": lane_peak,
                              "frac": lane_ops / lane_peak,
                              "lane_ops_per_update": FP32_LANE_OPS_PER_UPDATE_FF_2D,
                              "peak_source": f"bte_measure_peak(BTE_PEAK_FP32X2_FMA), measured at "
                                             f"{peaks_lib['sm_mhz']} MHz"},
                "fp64_fma_peak_flops": peaks_lib["fp64_fma_flops"]}
    variants = paper_TL100 = None
    if world == 1 and not args.no_variants:
        variants = run_variants(peaks, peaks_lib["fp64_fma_flops"])
        pd20, paper_TL100 = run_paper_device_20us(peaks)
        variants.append(pd20)
        variants.append(run_gs_variant(peaks, peaks_lib["fp64_fma_flops"]))
        variants.append(run_umesh_variant(peaks, peaks_lib["fp64_fma_flops"]))
        variants.append(run_umesh_variant(peaks, peaks_lib["fp64_fma_flops"], 1))
    cpu = accuracy = None
    if world == 1 and not args.no_cpu_baseline:
        ost, cpu = cpu_baseline_for(args, paper_TL100)
        accuracy = {"max_abs_dTL_K": float(np.max(np.abs(TL_first - ost["TL"]))),
                    "max_rel_dTL": float(np.max(np.abs(TL_first - ost["TL"]) / ost["TL"])),
                    "against": f"FP64 oracle, full {args.nx}x{args.ny} grid, first time step x {args.ninner} "
                               "inner iterations, same launch configuration as the timed steps"}
        del ost
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
           "scaling": "strong" if partitioned else "weak",
           "vs_baseline": None, "dtype": "f64 storage, double-float (f32x2) sweep arithmetic", "data": "synthetic",
           "config": workload_config(args, world, partitioned),
           "launch": ("CUDA graph per time step, autotuned (cells_per_cta,threads,grid,min_ctas_variant,directions_per_step): "
                      + tune_choice) if (tuned and not partitioned) else
                     ("eager launches (band-range exchange on the host between launches), " + tune_choice),
           "l2": "inputs larger than L2 (three FP64 intensity buffers of %.2f GB each)" % (wl.dof * 8 / 1e9),
           "gpu_launches": launches, "clocks": clk, "roofline": roofline, "e2e": e2e, "cpu_baseline": cpu,
           "accuracy": accuracy, "peaks_measured": peaks_lib, "variants": variants}
    if partitioned:
        out["band_ranges"] = [[r * wl.bands.nb // world, (r + 1) * wl.bands.nb // world] for r in range(world)]
        out["dist_backend"] = args.dist_backend
    print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
