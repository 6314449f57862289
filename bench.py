"""Benchmark: ensemble local-inertial flood model + particle filter on GB300.

Workload: 2000 x 2000 cells of 3 m (4.0 M cells), 96 members, triangular
60 mm/h storm peaking at 20 min, per-member rain multiplier LN(0, 0.3) and
Manning scale U[0.6, 1.4], six depth gauges observing a hidden truth member
with N(0, 0.05 m) noise.  One benchmark step = one 300 s assimilation window:
every member advances 300 s with its own CFL time step (fused flux +
continuity kernel, one launch per step for all members), then the gauges are
sampled and the particle filter weights, resamples and replaces members on
the device.  Twelve steps cover the 1 h storm.

Metric: member-cell-steps/s (members x cells x steps actually taken, per
second), plus the step kernel's HBM roofline fraction.

`--impl reference` times the FP64 CPU oracle (the reference for this
workload) on the host cores, each step a bounded sample of the same work.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

NY = NX = 2000
M = 96
ROWS = None
G = 6
WINDOW = 300.0
SEED = 1
BYTES_STATE = 24.0          # read + write h, qx, qy (FP32) per member-cell-step
BYTES_STATIC = 8.0          # z, n (FP32) per cell per tile pass
MEMBERS_PER_TILE = 4        # members sharing one static-field tile pass
ALGO_BYTES = BYTES_STATE + BYTES_STATIC / MEMBERS_PER_TILE
KERNEL_SOURCES = ["paper_2302_08341_gb300/csrc/step_kernel.cu",
                  "paper_2302_08341_gb300/csrc/step_tma.cu",
                  "paper_2302_08341_gb300/csrc/tma.cuh",
                  "paper_2302_08341_gb300/csrc/march.cuh",
                  "paper_2302_08341_gb300/csrc/tma_march.cuh",
                  "paper_2302_08341_gb300/csrc/flood_internal.cuh"]
BYTES_SINGLE = BYTES_STATE + BYTES_STATIC  # one member per static-field pass


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=12)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--ny", type=int, default=2000, help="rows (smaller cases for profiling)")
    ap.add_argument("--nx", type=int, default=2000)
    ap.add_argument("--members", type=int, default=96)
    ap.add_argument("--no-extensions", action="store_true",
                    help="skip the adjoint and uneven-batch measurements")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the default launch configuration (profiling runs)")
    ap.add_argument("--only", choices=["adjoint", "batch", "batch_land_cover", "calibration",
                                       "land_cover", "masked_domain", "products"],
                    help="run one extension measurement alone and print it (profiling runs)")
    ap.add_argument("--calibration-windows", type=int, default=3)
    ap.add_argument("--rows-per-strip", type=int, default=None,
                    help="strip height for --only calibration and --only batch")
    ap.add_argument("--engine", type=int, choices=[0, 1, 2], default=None,
                    help="step-kernel engine for --only batch (default: the library's)")
    args = ap.parse_args()
    global NY, NX, M, ROWS
    NY, NX, M, ROWS = args.ny, args.nx, args.members, args.rows_per_strip
    return args


def guarded(fn, *a, **kw):
    """Run one extension measurement; a failure is reported on the line
    instead of ending the run."""
    try:
        return fn(*a, **kw)
    except Exception as e:  # noqa: BLE001
        return {"error": f"{type(e).__name__}: {e}"}


def rounded(o, digits=4):
    """Floats of a nested result to `digits` significant digits (the
    extension figures; the timing keys keep full precision)."""
    if isinstance(o, float):
        return float(f"{o:.{digits}g}")
    if isinstance(o, dict):
        return {k: rounded(v, digits) for k, v in o.items()}
    if isinstance(o, list):
        return [rounded(v, digits) for v in o]
    return o


# (summary key, path into the extensions) of the figures repeated, compact,
# at the end of the line
SUMMARY_PATHS = [
    ("adj_over_fwd_1024x1024x1_1800s", ("adjoint", "adj_over_fwd")),
    ("adj_over_fwd_2000x2000x96_calibration", ("calibration", "adj_over_fwd")),
    ("adj_over_fwd_2000x2000x96_land_cover", ("land_cover", "adjoint", "adj_over_fwd")),
    ("calibration_ms_per_window", ("calibration", "ms_per_window")),
    ("batched_value", ("batched", "value")),
    ("batched_hbm_frac", ("batched", "hbm_frac_whole_window")),
    ("batched_persistent_value", ("batched", "persistent", "value")),
    ("batched_four_members_value", ("batched", "four_members", "value")),
    ("batched_four_members_hbm_frac", ("batched", "four_members", "hbm_frac_whole_window")),
    ("batched_land_cover_active_value", ("batched", "land_cover", "active_value")),
    ("land_cover_step_ms", ("land_cover", "step_kernel_ms")),
    ("land_cover_step_ms_without", ("land_cover", "without", "step_kernel_ms")),
    ("masked_domain_step_time_ratio", ("masked_domain", "step_time_ratio")),
    ("masked_domain_tiles_launched_frac", ("masked_domain", "masked", "tiles_launched_frac")),
    ("fused_over_plain_per_member", ("plain_vs_fused", "fused_over_plain")),
    ("cfl_bound_value", ("cfl_bound", "value")),
    ("cfl_bound_hbm_frac", ("cfl_bound", "hbm_frac_step_kernel")),
    ("products_ms_equal_weights", ("products", "products_ms_equal_weights")),
    ("products_ms_unequal_weights", ("products", "products_ms_unequal_weights")),
    ("products_alu_frac_equal", ("products", "alu_roofline", "equal_weights", "frac")),
    ("products_alu_frac_unequal", ("products", "alu_roofline", "unequal_weights", "frac")),
    ("eta_bar_us_96_members", ("eta_bar", "members_per_device", "96", "eta_bar_us_per_member_step")),
    ("graphs_speedup_256x256x1", ("graphs", "small", "speedup")),
    ("graphs_speedup_2000x2000x96", ("graphs", "ensemble", "speedup")),
    ("pf_update_ms_resampling", ("assimilation_overhead", "resampling_ms")),
    ("gauge_rmse_prior_m", ("da_skill", "rmse_prior_m")),
    ("gauge_rmse_posterior_m", ("da_skill", "rmse_posterior_m")),
]


def extension_summary(ext):
    """The headline figure of each extension, in one short object (a long
    line's readers may keep only its end); missing ones are left out."""
    out = {}
    for name, path in SUMMARY_PATHS:
        v = ext
        for k in path:
            v = v.get(k) if isinstance(v, dict) else None
        if isinstance(v, (int, float)) and not isinstance(v, bool):
            out[name] = rounded(float(v))
    return out


def kernel_hash():
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def traffic_per_unit():
    """DRAM bytes per member-cell-step of the step kernel from the committed
    ncu summary, if it was taken on the current kernel source (the summary
    carries `kernel_sha:` and `dram_bytes_per_member_cell_step:` lines)."""
    path = os.path.join(ROOT, "profiles", "step_kernel_traffic.md")
    try:
        with open(path) as f:
            kv = dict(l.strip().strip("`").split(":", 1) for l in f
                      if l.strip().strip("`").split(":", 1)[0] in
                      ("kernel_sha", "dram_bytes_per_member_cell_step"))
    except (OSError, ValueError):
        return None
    if kv.get("kernel_sha", "").strip() != kernel_hash():
        return None
    try:
        return float(kv["dram_bytes_per_member_cell_step"])
    except (KeyError, ValueError):
        return None


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, ValueError, KeyError):
        return 6800.0, "fallback"


class Clocks:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.f = None

    def __enter__(self):
        try:
            self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, ValueError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.proc or not self.f:
            return None
        self.f.flush()
        rows = []
        with open(self.f.name) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
                except ValueError:
                    continue
        os.unlink(self.f.name)
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i, v in enumerate(r)
                          if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows),
                "sm_max_mhz": max(r[1] for r in rows), "reasons": reasons,
                "samples": len(rows)}


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(x, world, device):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x, world, device):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def job_value(units, ms, world, device):
    """Whole-job throughput: the units every rank processed over the slowest
    rank's time (weak scaling: each rank runs its own replica)."""
    ms_max = max_over_ranks(ms, world, device)
    units_all = sum_over_ranks(units, world, device)
    return units_all / (ms_max * 1e-3), ms_max


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def workload_config():
    """The benchmark workload, the same for both arms."""
    return {"workload": f"ensemble flood + particle filter: {NY}x{NX} cells (3 m), {M} members, "
                        "300 s assimilation windows, 1 h triangular storm",
            "cells": NY * NX, "members": M, "gauges": G, "window_s": WINDOW}


def make_inputs():
    from paper_2302_08341_gb300 import synth
    terr = synth.make_terrain(NY, NX, seed=SEED)
    hy = synth.hyetograph_triangular(60.0, 1200.0, 3600.0)
    rm, sc = synth.ensemble_prior(SEED, M)
    cells = synth.gauge_cells(terr, G, seed=SEED)
    return terr, hy, rm, sc, cells


def truth_observations(capi, terr, hy, cells, n_windows):
    """Hidden truth member (own prior draw) run on the GPU; noisy depths at
    the gauges at every window end (inputs of the benchmark, not timed), and
    the truth's own depths there."""
    from paper_2302_08341_gb300 import synth
    trm, tsc = synth.ensemble_prior(SEED + 1000, 1)
    obs, truth = [], []
    with capi.Grid(terr.z, terr.n) as g:
        g.ensemble_init(1, trm, tsc, hy)
        for w in range(1, n_windows + 1):
            g.advance_to(WINDOW * w)
            y = g.gauge_sample(cells)
            obs.append(synth.observe(y[0], seed=SEED, window=w))
            truth.append(y[0].astype(np.float64))
    return obs, np.array(truth)


def cpu_baseline(terr, hy, rm, sc, target_s=15.0):
    """The FP64 oracle on the host, single thread, on a bounded sample: one
    member of the 2000 x 2000 grid from a 5 cm wet start, as many steps as
    fit in ~target_s."""
    import oracle
    p = oracle.Params(ny=NY, nx=NX)
    z = terr.z.astype(np.float64); n = terr.n.astype(np.float64)
    m = oracle.Member.dry(NY, NX, np.full((NY, NX), 0.05))
    hy64 = hy.astype(np.float64)
    t0 = time.perf_counter()
    steps = 0
    while time.perf_counter() - t0 < target_s:
        oracle.advance(p, z, n, float(sc[0]), float(rm[0]), hy64, m, max_steps=2)
        steps += 2
    el = time.perf_counter() - t0
    return {"value": steps * NY * NX / el, "unit": "member-cell-steps/s", "cores": 1,
            "kind": "oracle",
            "sample": f"1 member x {NY}x{NX} cells x {steps} steps from a 5 cm wet start, "
                      f"FP64, 1 thread, {el:.1f} s"}


def cpu_all_cores(terr, hy, rm, sc, target_s=10.0):
    """The same oracle on every host core: one member per core, advanced
    together by the oracle's own ensemble loop (one thread per member), on a
    bounded sample from the same 5 cm wet start."""
    import oracle
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    cores = max(1, min(int(cores or 1), len(rm)))
    p = oracle.Params(ny=NY, nx=NX)
    z = terr.z.astype(np.float64); n = terr.n.astype(np.float64)
    e = oracle.Ensemble(p, cores, h0=np.full((NY, NX), 0.05))
    sc64 = sc[:cores].astype(np.float64); rm64 = rm[:cores].astype(np.float64)
    hy64 = hy.astype(np.float64)
    t0 = time.perf_counter()
    steps = 0
    while time.perf_counter() - t0 < target_s:
        steps += int(e.advance(z, n, sc64, rm64, hy64, max_steps=2, nthreads=cores).sum())
    el = time.perf_counter() - t0
    return {"value": steps * NY * NX / el, "unit": "member-cell-steps/s", "cores": cores,
            "kind": "oracle",
            "sample": f"{cores} members x {NY}x{NX} cells, {steps} member-steps from a 5 cm wet "
                      f"start, FP64, {cores} threads, {el:.1f} s"}


def adjoint_measure(capi):
    """Adjoint cost: 1024 x 1024 single member, 8 gauges sampled every 60 s over
    1800 s, checkpoint every 64 steps; reverse (replay included) / forward."""
    from paper_2302_08341_gb300 import synth
    terr = synth.make_terrain(1024, 1024, seed=3)
    hy = synth.hyetograph_triangular(60.0, 1200.0, 3600.0)
    rm, sc = synth.ensemble_prior(3, 1)
    cells = synth.gauge_cells(terr, 8, seed=3)
    trm, tsc = synth.ensemble_prior(1003, 1)
    obs = []
    with capi.Grid(terr.z, terr.n) as g:
        g.ensemble_init(1, trm, tsc, hy)
        for s in range(1, 31):
            g.advance_to(60.0 * s)
            obs.append(synth.observe(g.gauge_sample(cells)[0], seed=3, window=s))
    d = np.array(obs)
    res = None
    with capi.Grid(terr.z, terr.n) as g:
        for _ in range(2):  # the first call sizes the buffers
            g.ensemble_init(1, rm, sc, hy)
            res = g.adjoint(cells, d, 60.0, ckpt_every=64)
    return {"config": "1024x1024 cells, 1 member, 8 gauges every 60 s over 1800 s, "
                      "checkpoint every 64 steps",
            "forward_ms": res["forward_ms"], "reverse_ms": res["reverse_ms"],
            "adj_over_fwd": res["reverse_ms"] / res["forward_ms"]}


def batch_measure(capi, engine=None, rows=None, tune=False, members=1, land_cover=False):
    """Uneven batch: 64 scenarios, square sides U{512..2048}, own DEM seeds,
    rain U[20, 100] mm/h, durations U[900, 3600] s, advanced in 300 s windows
    by graph-replayed batched launches; member-cell-steps/s over the batch.
    members > 1: that many members per scenario (rain multiplier LN(0, 0.3),
    Manning scale U[0.6, 1.4] each), sharing the scenario's bed and
    roughness tile by tile.  land_cover: every scenario with its own land
    cover (Section 4.1: roads and buildings hardened and drained, ponds,
    green land, two corners outside the domain) and each member with its
    own class roughness and drainage rate."""
    import torch
    from paper_2302_08341_gb300 import synth
    scen = synth.uneven_batch(64)
    terrs = [synth.make_terrain(s.ny, s.nx, seed=s.seed) for s in scen]
    clss = [synth.land_cover(t, seed=s.seed) for t, s in zip(terrs, scen)] if land_cover else None
    hys = [synth.hyetograph_constant(s.rain_mm_h, s.duration_s) for s in scen]
    dur = np.array([s.duration_s for s in scen])
    counts = np.full(len(scen), members, np.int32)
    if members > 1:
        rm, sc = synth.ensemble_prior(SEED + 64, int(counts.sum()))
    else:
        rm = sc = np.ones(len(scen), np.float32)
    mkw = {"members": counts} if members > 1 else {}
    cells = np.repeat(np.array([s.ny * s.nx for s in scen], np.float64), counts)
    first = np.concatenate([[0], np.cumsum(counts)])
    if land_cover:
        outside = np.array([c[3] for c in synth.LAND_CLASSES], bool)
        active = np.repeat(np.array([float((~outside[c]).sum()) for c in clss]), counts)
        n_m, d_m = synth.land_prior(SEED + 65, int(counts.sum()))
    dur_m = np.repeat(dur, counts)
    tuned = None

    def init(b):
        b.init(hys, rm, sc, dur, **mkw)
        if land_cover:
            for i in range(len(scen)):
                b.set_land_params(i, n_m[first[i]:first[i + 1]], d_m[first[i]:first[i + 1]])

    with capi.Batch([t.z for t in terrs], [t.n for t in terrs]) as b:
        if land_cover:
            for i, c in enumerate(clss):
                b.set_land_cover(i, c, synth.LAND_CLASSES)
        if engine is not None:
            b.set_engine(engine)
        else:
            engine = 1
        rows = rows or ROWS
        if rows:
            b.set_launch(rows, 4)
        init(b)
        b.step(300.0)                      # warm-up window (graph capture)
        if tune:                           # on the live batch after the first window
            r, w, e, t = b.autotune(30.0)
            tuned = {"rows_per_strip": r, "warps_per_cta": w, "engine": e, "trial_ms": t}
            engine, rows = e, r
        init(b)
        stream = torch.cuda.current_stream()
        e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
        l0 = b.launch_count
        torch.cuda.synchronize()
        e0.record(stream)
        for w in range(1, 13):
            b.step(300.0 * w, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        mem = b.members()
        launches = b.launch_count - l0
    units = float((mem["steps"] * cells).sum())
    extra = {}
    if land_cover:
        extra = {"land_cover": "4 classes per scenario, per-member class roughness and drainage",
                 "active_value": float((mem["steps"] * active).sum()) / (ms * 1e-3),
                 "active_frac": float(active.sum() / cells.sum())}
    form = {0: "direct loads, CUDA-graph replayed per-step launches",
            1: "TMA-staged rows, CUDA-graph replayed per-step launches",
            2: "TMA-staged rows, one persistent cooperative launch per window"}[engine]
    return {"config": "64 scenarios, sides U{512..2048}, rain U[20,100] mm/h, durations "
                      f"U[900,3600] s, {members} member(s) each, 300 s windows, batched step: "
                      + form,
            "value": units / (ms * 1e-3), "unit": "member-cell-steps/s", "ms": ms,
            "members_per_scenario": members,
            "total_cells": float(cells.sum()), "member_cell_steps": units,
            "all_finished": bool(np.all(mem["t"] == dur_m)), "gpu_launches": launches,
            "engine": {0: "direct loads", 1: "tma", 2: "tma persistent"}[engine],
            "engine_id": engine,
            "rows_per_strip": rows or 64, "autotune": tuned, **extra}


def calibration_measure(capi, windows=3):
    """Ensemble gradient calibration + particle filter: 2000 x 2000 cells, 96
    members, a shared 64 x 64 roughness factor field over the base Manning
    field.  Per 300 s window: the adjoint of the window (loss: squared misfit
    of the 6 gauges at its end, summed over members), one calibration step
    on the rain multipliers and the field, then the gauge sample and the
    particle filter.  The first window sizes the adjoint's buffers (about
    190 GB of checkpoints and replay states) and is not counted."""
    import torch
    from paper_2302_08341_gb300 import synth
    terr = synth.make_terrain(NY, NX, seed=4)
    hy = synth.hyetograph_triangular(60.0, 1200.0, 3600.0)
    rm, sc = synth.ensemble_prior(4, M)
    cells = synth.gauge_cells(terr, G, seed=4)
    trm, tsc = synth.ensemble_prior(1004, 1)
    obs = []
    with capi.Grid(terr.z, terr.n) as t:
        t.ensemble_init(1, trm, tsc, hy)
        for w in range(1, windows + 1):
            t.advance_to(WINDOW * w)
            obs.append(synth.observe(t.gauge_sample(cells)[0], seed=4, window=w))
    stream = torch.cuda.current_stream()
    rows = []
    with capi.Grid(terr.z, terr.n) as g:
        g.ensemble_init(M, rm, sc, hy, stream=stream)
        g.set_roughness_factor(np.ones((64, 64), np.float32), stream=stream)
        if ROWS:
            g.set_launch(ROWS, 4 if M >= 4 else 1)
        for w in range(1, windows + 1):
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
            s0 = g.members()["steps"].sum()
            torch.cuda.synchronize()
            ev[0].record(stream)
            out = g.adjoint(cells, obs[w - 1][None, :], WINDOW, grad_h0=False, stream=stream)
            ev[1].record(stream)
            loss = g.calibration_step(stream=stream)
            ev[2].record(stream)
            u, beta = synth.pf_draws(4, w, M)
            g.gauge_sample(cells, stream=stream)
            pf = g.pf_assimilate(obs[w - 1], 0.05, u, beta, stream=stream)
            ev[3].record(stream)
            torch.cuda.synchronize()
            member_steps = float(g.members()["steps"].sum() - s0)
            rows.append({"window_ms": ev[0].elapsed_time(ev[3]),
                         "adjoint_ms": ev[0].elapsed_time(ev[1]),
                         "adjoint_forward_ms": out["forward_ms"],
                         "adjoint_reverse_ms": out["reverse_ms"],
                         "calibration_step_ms": ev[1].elapsed_time(ev[2]),
                         "pf_ms": ev[2].elapsed_time(ev[3]),
                         "loss": float(np.sum(loss)), "neff": float(pf["neff"]),
                         "member_cell_steps": member_steps * NY * NX})
    timed = rows[1:] if len(rows) > 1 else rows
    avg = {k: float(np.mean([r[k] for r in timed])) for k in timed[0]}
    return {"config": f"{NY}x{NX} cells, {M} members, 64x64 roughness factor field, 6 gauges, "
                      f"{len(timed)} timed 300 s windows after one that sizes the buffers",
            "ms_per_window": avg["window_ms"], "adjoint_ms": avg["adjoint_ms"],
            "adjoint_forward_ms": avg["adjoint_forward_ms"],
            "adjoint_reverse_ms": avg["adjoint_reverse_ms"],
            "adj_over_fwd": avg["adjoint_reverse_ms"] / avg["adjoint_forward_ms"],
            "calibration_step_ms": avg["calibration_step_ms"], "pf_ms": avg["pf_ms"],
            "forward_member_cell_steps_per_s": avg["member_cell_steps"] /
            (avg["adjoint_forward_ms"] * 1e-3),
            "loss_by_window": [r["loss"] for r in rows], "neff_by_window": [r["neff"] for r in rows]}


def plain_vs_fused(g, tuned, stream, device, ncell, hbm_peak):
    """The same ensemble advanced one 300 s window by the fused ensemble step
    (one launch per step for all members) and the next window by the plain
    form (one launch per member per step, bed and roughness read per member,
    with the strip height that suits a single member picked by a short
    sweep); member-cell-steps/s of each on this GPU."""
    import torch
    fused_engine = tuned["engine"] if tuned else 1
    fused_shape = (tuned["rows_per_strip"], tuned["members_per_cta"]) if tuned else (0, 0)
    t = float(g.members()["t"].max())

    def timed(span):
        nonlocal t
        s0 = g.members()["steps"].sum()
        l0 = g.launch_count
        e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(device)
        e0.record(stream)
        t += span
        g.advance_to(t, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize(device)
        ms = e0.elapsed_time(e1)
        units = float(g.members()["steps"].sum() - s0) * ncell
        return units / (ms * 1e-3), ms, g.launch_count - l0

    out = {}
    g.set_engine(2)
    sweep = {}
    for rows in (4, 8, 16, 32):
        g.set_launch(rows, 1)
        sweep[rows] = timed(10.0)[0]
    plain_rows = max(sweep, key=sweep.get)
    for name, eng, shape, nbytes in (("fused", fused_engine, fused_shape, ALGO_BYTES),
                                     ("plain_per_member", 2, (plain_rows, 1), BYTES_SINGLE)):
        g.set_engine(eng)
        g.set_launch(*shape)
        v, ms, launches = timed(WINDOW)
        out[name] = {"value": v, "unit": "member-cell-steps/s", "ms_per_window": ms,
                     "gpu_launches": launches, "rows_per_strip": shape[0],
                     "algorithmic_bytes_per_member_cell_step": nbytes,
                     "hbm_frac_whole_window": v * nbytes / 1e9 / hbm_peak}
    out["plain_rows_sweep"] = {str(k): v for k, v in sweep.items()}
    g.set_engine(fused_engine)
    g.set_launch(*fused_shape)
    out["fused_over_plain"] = out["fused"]["value"] / out["plain_per_member"]["value"]
    out["config"] = "one 300 s window each, after the timed windows, no particle filter"
    return out


def cfl_bound_measure(capi, terr, hy, rm, sc, tuned):
    """The benchmark's hour never lets Eq. 4 bind (its depths stay under the
    0.45 m at which 0.7 dx / sqrt(g h) falls below the 1 s cap).  Here the
    same 96 members start from 1 m of water with five times the storm, so
    every member steps at its own CFL-limited dt (about 0.6-0.7 s) and the
    members' clocks drift apart between window ends; one 300 s window is
    timed after a 60 s warm-up."""
    import torch
    stream = torch.cuda.current_stream()
    h0 = np.full(terr.z.shape, 1.0, np.float32)
    with capi.Grid(terr.z, terr.n) as g:
        g.ensemble_init(M, (rm * 5.0).astype(np.float32), sc, hy, h0=h0, stream=stream)
        if tuned:
            g.set_engine(tuned["engine"])
            g.set_launch(tuned["rows_per_strip"], tuned["members_per_cta"])
        g.advance_to(60.0, stream=stream)
        m0 = g.members()
        g.profile(True)
        e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        g.advance_to(60.0 + WINDOW, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        kms, kn = g.profile(False)
        m1 = g.members()
    steps = m1["steps"] - m0["steps"]
    ms = e0.elapsed_time(e1)
    units = float(steps.sum()) * terr.z.size
    return {"config": f"{terr.z.shape[0]}x{terr.z.shape[1]} cells, {M} members from 1 m of water, "
                      "5x the storm, one 300 s window with Eq. 4 binding",
            "value": units / (ms * 1e-3), "unit": "member-cell-steps/s", "ms_per_window": ms,
            "step_kernel_ms": kms / max(kn, 1), "step_launches": int(kn),
            "member_steps_min": int(steps.min()), "member_steps_max": int(steps.max()),
            "mean_dt_s": WINDOW * M / float(steps.sum()),
            "hbm_frac_step_kernel": float(steps.sum()) * terr.z.size * ALGO_BYTES
                                    / (kms * 1e-3) / 1e9 / peaks()[0]}


def graphs_measure(capi, terr, hy, rm, sc, tuned):
    """The ensemble's steps launched one by one against runs of 24 steps
    replayed from a CUDA graph (flood_set_graphs), both timed with CUDA
    events around one flood_step call: a small single-member grid whose
    kernels last microseconds (256 x 256 cells, 50 mm/h, 600 s of steps: the
    launches bound it), and one 300 s window of the benchmark ensemble (the
    step kernel bounds it).  The capture of each call's run is inside the
    timed region."""
    import torch
    from paper_2302_08341_gb300 import synth
    stream = torch.cuda.current_stream()
    small = synth.make_terrain(256, 256, seed=0)
    cases = {"small": (small, synth.hyetograph_constant(50.0, 900.0),
                       np.ones(1, np.float32), np.ones(1, np.float32), 30.0, 630.0, None),
             "ensemble": (terr, hy, rm, sc, 60.0, 60.0 + WINDOW, tuned)}
    res = {}
    for name, (tr, hyc, rmc, scc, t0, t1, tun) in cases.items():
        out = {}
        for graphs in (False, True):
            with capi.Grid(tr.z, tr.n) as g:
                g.ensemble_init(len(rmc), rmc, scc, hyc, stream=stream)
                if tun:
                    g.set_engine(tun["engine"])
                    g.set_launch(tun["rows_per_strip"], tun["members_per_cta"])
                g.set_graphs(graphs)
                g.advance_to(t0, stream=stream)
                s0 = g.members()["steps"].sum()
                e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
                torch.cuda.synchronize()
                h0 = time.perf_counter()
                e0.record(stream)
                g.advance_to(t1, stream=stream)
                e1.record(stream)
                torch.cuda.synchronize()
                wall = (time.perf_counter() - h0) * 1e3
                steps = float(g.members()["steps"].sum() - s0)
                out["graphs" if graphs else "plain"] = {
                    "ms": e0.elapsed_time(e1), "host_ms": wall,
                    "member_cell_steps_per_s": steps * tr.z.size / (e0.elapsed_time(e1) * 1e-3),
                    "captures_replays": list(g.graph_stats())}
        out["speedup"] = out["plain"]["ms"] / out["graphs"]["ms"]
        out["config"] = (f"{tr.z.shape[0]}x{tr.z.shape[1]} cells, {len(rmc)} member(s), "
                         f"flood_step from t = {t0:g} s to {t1:g} s")
        res[name] = out
    return res


def eta_sweeps(capi, g, tuned, stream, device, terr, hy, rm, sc):
    """Section 4.4's eta-bar (Eq. 13: the run time of one member, the
    ensemble's time divided by the members sharing the device) on this GPU,
    two ways: members per CTA (the paper's thread-block z-dimension, whose
    warps share one tile of the bed and roughness) on the live 96-member
    ensemble, and members on the device (a fresh ensemble of n members from
    a 5 cm wet start); 60 steps each, step-kernel time from CUDA events."""
    import torch
    rows = tuned["rows_per_strip"] if tuned else 0
    eng = tuned["engine"] if tuned else 1
    t = float(g.members()["t"].max())
    per_cta = {}
    g.set_engine(1)
    for mpc in (1, 2, 4, 8):
        g.set_launch(rows or 32, mpc)
        g.profile(True)
        t += 60.0
        s0 = g.members()["steps"].sum()
        g.advance_to(t, stream=stream)
        kms, kn = g.profile(False)
        steps = float(g.members()["steps"].sum() - s0)
        per_cta[str(mpc)] = {"ms_per_step": kms / max(kn, 1),
                             "eta_bar_us_per_member_step": kms / max(steps, 1) * 1e3}
    g.set_engine(eng)
    g.set_launch(*((tuned["rows_per_strip"], tuned["members_per_cta"]) if tuned else (0, 0)))
    per_device = {}
    for n in (1, 2, 4, 8, 16, 32, 64, 96):
        with capi.Grid(terr.z, terr.n) as e:
            e.ensemble_init(n, rm[:n], sc[:n], hy, h0=np.full(terr.z.shape, 0.05, np.float32),
                            stream=stream)
            e.advance_to(10.0, stream=stream)          # warm-up
            e.profile(True)
            s0 = e.members()["steps"].sum()
            e.advance_to(70.0, stream=stream)
            kms, kn = e.profile(False)
            steps = float(e.members()["steps"].sum() - s0)
            per_device[str(n)] = {"ms_per_step": kms / max(kn, 1),
                                  "eta_bar_us_per_member_step": kms / max(steps, 1) * 1e3}
    best = min(per_cta, key=lambda k: per_cta[k]["eta_bar_us_per_member_step"])
    return {"config": "eta-bar = step-kernel time / member-steps (Eq. 13 per step); members per "
                      "CTA on the live 96-member ensemble; members on the device from a 5 cm wet "
                      "start", "members_per_cta": per_cta, "members_per_device": per_device,
            "best_members_per_cta": int(best),
            "per_cta_gain_best_over_1": per_cta["1"]["eta_bar_us_per_member_step"]
                                        / per_cta[best]["eta_bar_us_per_member_step"] - 1.0}


def products_only(capi):
    """The product maps alone (profiling): an ensemble of the benchmark's
    shape with its running maxima tracked over 60 s from a 5 cm wet start,
    then the exceedance and 10/50/90 % maps three times with equal weights
    and three times with unequal ones, maps kept on the device."""
    import torch
    from paper_2302_08341_gb300 import synth
    device = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(device)
    terr = synth.make_terrain(NY, NX, seed=SEED)
    hy = synth.hyetograph_triangular(60.0, 1200.0, 3600.0)
    rm, sc = synth.ensemble_prior(SEED, M)
    maps = (torch.empty((NY, NX), dtype=torch.float32, device=device),
            torch.empty((3, NY, NX), dtype=torch.float32, device=device))
    res = {}
    with capi.Grid(terr.z, terr.n) as g:
        g.ensemble_init(M, rm, sc, hy, h0=np.full((NY, NX), 0.05, np.float32), stream=stream)
        g.track_max_depth(True, stream=stream)
        g.advance_to(60.0, stream=stream)
        for name, w in (("equal_weights", np.full(M, 1.0 / M)),
                        ("unequal_weights", np.linspace(1.0, 3.0, M) / np.linspace(1.0, 3.0, M).sum())):
            g.set_members(weights=w)
            ts = []
            for _ in range(3):
                e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                g.ensemble_products(0.2, (0.1, 0.5, 0.9), stream=stream, out=maps)
                e1.record(stream)
                torch.cuda.synchronize(device)
                ts.append(e0.elapsed_time(e1))
            res[name + "_ms"] = ts
    return res


def assimilation_overhead(g, stream, device, cells, obs):
    """Fig. 12c's analogue: one assimilation round (gauge sample, weights,
    N_eff, and -- when resampling -- the systematic resampling, the member
    copies and the perturbation) on the 96-member 4.0 M-cell ensemble, timed
    by CUDA events with and without resampling (5 rounds each)."""
    import torch
    from paper_2302_08341_gb300 import synth
    M_ = g.M
    out = {}
    for name, force, thr in (("no_resampling", False, 0.0), ("resampling", True, 0.8)):
        ts = []
        for r in range(5):
            u, beta = synth.pf_draws(SEED, 100 + r, M_)
            e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize(device)
            e0.record(stream)
            g.gauge_sample(cells, stream=stream)
            pf = g.pf_assimilate(obs, 0.05, u, beta, stream=stream, force=force, n_thr_frac=thr)
            e1.record(stream)
            torch.cuda.synchronize(device)
            ts.append(e0.elapsed_time(e1))
            assert bool(pf["resampled"]) == force
        out[name + "_ms"] = float(np.median(ts))
    out["resampling_over_no_resampling"] = out["resampling_ms"] / out["no_resampling_ms"]
    out["config"] = ("gauge sample + particle-filter update of 96 members x 4.0 M cells, median "
                     "of 5 rounds; the call includes the host reading the filter's outputs")
    return out


def land_cover_measure(capi):
    """Land cover (Section 4.1) on the benchmark ensemble: 2000 x 2000 cells,
    96 members with their own class roughness (Table 1 ranges) and drainage
    rate, green land / water / hardened ground / cells outside the domain;
    the second 300 s window of the storm is timed (the first warms up)."""
    import torch
    from paper_2302_08341_gb300 import synth
    terr = synth.make_terrain(NY, NX, seed=SEED)
    cls = synth.land_cover(terr, seed=SEED)
    hy = synth.hyetograph_triangular(60.0, 1200.0, 3600.0)
    rm, sc = synth.ensemble_prior(SEED, M)
    n_m, d_m = synth.land_prior(SEED, M)
    stream = torch.cuda.current_stream()
    res = {}
    for name, land in (("land_cover", True), ("same_window_without", False)):
        with capi.Grid(terr.z, terr.n) as g:
            if land:
                g.set_land_cover(cls, synth.LAND_CLASSES)
            g.ensemble_init(M, rm, sc, hy, stream=stream)
            if land:
                g.set_land_params(n_m, d_m)
            g.profile(True)
            g.advance_to(WINDOW, stream=stream)
            g.profile(False)
            tuned = g.autotune(steps_per_trial=6, stream=stream)   # the ensemble is left as it was
            g.profile(True)
            s0 = g.members()["steps"].sum()
            e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            g.advance_to(2 * WINDOW, stream=stream)
            e1.record(stream)
            torch.cuda.synchronize()
            kms, kn = g.profile(False)
            ms = e0.elapsed_time(e1)
            # only the cells of the domain count as work (the outside ones carry none)
            active = float((cls != 3).sum()) if land else float(NY * NX)
            units = float(g.members()["steps"].sum() - s0) * active
            res[name] = {"value": units / (ms * 1e-3), "ms_per_window": ms,
                         "step_kernel_ms": kms / max(kn, 1), "active_cells": active,
                         "autotune": {"rows_per_strip": tuned[0], "members_per_cta": tuned[1],
                                      "engine": tuned[2], "ms_per_step": tuned[3]}}
            if land:
                vol = g.volumes()
                drained = g.drained()
                # the adjoint across land cover: the third window against 6
                # gauges sampled every 60 s
                cells = synth.gauge_cells(terr, 6, seed=SEED)
                cells = cells[cls.ravel()[cells] != 3]
                obs = np.full((5, len(cells)), 0.1)
                if ROWS:
                    g.set_launch(ROWS, 4 if M >= 4 else 1)
                out = g.adjoint(cells, obs, 60.0, stream=stream)
                _, gd = g.adjoint_land_grad()
                adj = {"window_s": 300.0, "gauges": int(len(cells)),
                       "forward_ms": out["forward_ms"], "reverse_ms": out["reverse_ms"],
                       "adj_over_fwd": out["reverse_ms"] / max(out["forward_ms"], 1e-9),
                       "drain_grad_finite": bool(np.all(np.isfinite(gd)))}
    return {"config": f"{NY}x{NX} cells, {M} members, 4 land classes "
                      f"({100 * (cls == 3).mean():.1f} % of the cells outside the domain), "
                      "second 300 s window, against the same window without land cover",
            "value": res["land_cover"]["value"], "unit": "member-cell-steps/s",
            "ms_per_window": res["land_cover"]["ms_per_window"],
            "step_kernel_ms": res["land_cover"]["step_kernel_ms"],
            "without": res["same_window_without"],
            "drained_share_of_rain": float(np.mean(drained / vol["rain"])),
            "adjoint": adj}


def masked_domain_measure(capi):
    """Land cover over an irregular domain shaped like the paper's study area
    (Section 4.1: 4,002,457 active cells of 3 m in an 8.2 x 7.6 km box):
    2533 x 2733 cells, 57.8 % active (4.0 M), 96 members.  The step launches
    only the tiles that hold a cell of the domain; beside it, the same box
    with every cell active.  Member-cell-steps count active cells only; the
    second 300 s window is timed."""
    import torch
    from paper_2302_08341_gb300 import synth
    ny, nx = 2533, 2733
    terr = synth.make_terrain(ny, nx, seed=SEED)
    dom = synth.irregular_domain(ny, nx, 0.578, seed=SEED)
    hy = synth.hyetograph_triangular(60.0, 1200.0, 3600.0)
    rm, sc = synth.ensemble_prior(SEED, M)
    n_m, d_m = synth.land_prior(SEED, M)
    stream = torch.cuda.current_stream()
    res = {}
    for name, domain in (("masked", dom), ("whole_box", np.ones_like(dom))):
        cls = synth.land_cover(terr, seed=SEED, domain=domain)
        active = float(domain.sum())
        with capi.Grid(terr.z, terr.n) as g:
            g.set_land_cover(cls, synth.LAND_CLASSES)
            g.ensemble_init(M, rm, sc, hy, stream=stream)
            g.set_land_params(n_m, d_m)
            g.advance_to(WINDOW, stream=stream)
            rows, _ = g.get_launch()
            g.profile(True)
            s0 = g.members()["steps"].sum()
            e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            g.advance_to(2 * WINDOW, stream=stream)
            e1.record(stream)
            torch.cuda.synchronize()
            kms, kn = g.profile(False)
            ms = e0.elapsed_time(e1)
            steps = float(g.members()["steps"].sum() - s0)
        tiles = sum(bool(domain[a:a + rows, b:b + 128].any())
                    for a in range(0, ny, rows) for b in range(0, nx, 128))
        tiles_all = ((ny + rows - 1) // rows) * ((nx + 127) // 128)
        step_ms = kms / max(kn, 1)
        # algorithmic bytes: 26 B per active member-cell-step (26.25 B with the class byte)
        res[name] = {"value": steps * active / (ms * 1e-3), "unit": "member-cell-steps/s",
                     "active_cells": active, "active_frac": active / (ny * nx),
                     "tiles_launched_frac": tiles / tiles_all, "rows_per_strip": rows,
                     "ms_per_window": ms, "step_kernel_ms": step_ms,
                     "hbm_frac_active": steps / max(kn, 1) * active * 26.25 / (step_ms * 1e-3)
                                        / 1e9 / peaks()[0]}
    res["config"] = (f"{ny}x{nx} box, {M} members, land cover, irregular domain "
                     f"{100 * dom.mean():.1f} % active ({int(dom.sum())} cells), second 300 s window")
    res["step_time_ratio"] = res["masked"]["step_kernel_ms"] / res["whole_box"]["step_kernel_ms"]
    return res


def sort_network(M):
    """The comparators (lo, hi) of the products kernels' register sort, in
    order: Batcher's odd-even merge sort on N (a power of two) slots with
    every comparator that reaches a padding slot at or above MT left out
    (MT = the member count rounded up to 32, 64, 96 or 128; N = MT rounded up
    to a power of two), the same pruning rule as the kernels.  The padding
    slots hold +inf, so the comparators left out never move a value."""
    MT = 32 if M <= 32 else 64 if M <= 64 else 96 if M <= 96 else 128
    N = 32 if MT <= 32 else 64 if MT <= 64 else 128
    pairs, P = [], 1
    while P < N:
        K = P
        while K >= 1:
            j = K % P
            while j + K < N:
                pairs += [(i + j, i + j + K) for i in range(K)
                          if i + j + K < MT and (i + j) // (2 * P) == (i + j + K) // (2 * P)]
                j += 2 * K
            K //= 2
        P *= 2
    return pairs


def network_minmax(M):
    """Min/max operations per cell of the products kernels' register sort:
    two per comparator of `sort_network` (1056 comparators at 96 members)."""
    return 2 * len(sort_network(M))


# Minimum / maximum results per clock per SM (the ALU pipe: 16 lanes per
# scheduler, 4 schedulers).
ALU_MINMAX_PER_CLK_SM = 64


def alu_roofline(ops, ms, sm_mhz):
    """The sort network's min/max operations per second against the ALU
    pipe's peak at the sampled SM clock, over the device's SMs."""
    import torch
    n_sm = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    peak = ALU_MINMAX_PER_CLK_SM * n_sm * sm_mhz * 1e6
    achieved = ops / (ms * 1e-3)
    return {"bound": "alu", "achieved": achieved / 1e12, "peak": peak / 1e12,
            "unit": "T min/max per s", "frac": achieved / peak, "ops_per_cell": ops / (NY * NX),
            "sms": n_sm}


def products_measure(g, stream, device, ncell, fused_value):
    """Section 4.4's products on the benchmark ensemble: one 300 s window with
    every member's running maximum depth kept by the step kernel (8 more
    bytes per member-cell-step), then the exceedance map P(hmax >= 0.2 m)
    and the 10/50/90 % maps of the maximum depth over the weighted ensemble."""
    import torch
    t = float(g.members()["t"].max())
    g.track_max_depth(True, stream=stream)
    s0 = g.members()["steps"].sum()
    e = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    torch.cuda.synchronize(device)
    e[0].record(stream)
    g.advance_to(t + WINDOW, stream=stream)
    e[1].record(stream)
    torch.cuda.synchronize(device)
    units = float(g.members()["steps"].sum() - s0) * ncell
    w0 = g.members()["weights"]

    maps = (torch.empty((NY, NX), dtype=torch.float32, device=device),
            torch.empty((3, NY, NX), dtype=torch.float32, device=device))

    def timed_products():
        # the call is synchronous; the events bracket it on the same stream,
        # the maps stay on the device
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ev[0].record(stream)
        ex, _ = g.ensemble_products(0.2, (0.1, 0.5, 0.9), stream=stream, out=maps)
        ev[1].record(stream)
        torch.cuda.synchronize(device)
        return ev[0].elapsed_time(ev[1]), ex.cpu().numpy()

    g.set_members(weights=np.full(len(w0), 1.0 / len(w0)))
    timed_products()                                  # first call: allocator, attributes
    eq_ms, exceed = timed_products()
    wu = np.linspace(1.0, 3.0, len(w0)); wu /= wu.sum()
    g.set_members(weights=wu)
    uneq_ms, _ = timed_products()
    g.set_members(weights=w0)
    cur_ms, _ = timed_products()
    g.track_max_depth(False, stream=stream)
    v = units / (e[0].elapsed_time(e[1]) * 1e-3)
    maxima_bytes = float(len(w0)) * ncell * 4.0 + 4.0 * ncell * 4.0   # maxima in, 4 maps out
    return {"config": "one 300 s window with the running maxima tracked, then P(hmax >= 0.2 m) "
                      "and the 10/50/90 % maps over 96 members (4.0 M cells each)",
            "tracked_value": v, "unit": "member-cell-steps/s",
            "tracking_cost": fused_value / v - 1.0,
            "products_ms": cur_ms,
            "weights_equal_after_filter": bool(np.all(w0 == w0[0])),
            "products_ms_equal_weights": eq_ms,
            "products_ms_unequal_weights": uneq_ms,
            "products_hbm_frac_equal_weights": maxima_bytes / (eq_ms * 1e-3) / 1e9 / peaks()[0],
            "products_hbm_frac_unequal_weights": maxima_bytes / (uneq_ms * 1e-3) / 1e9 / peaks()[0],
            "network_ops": float(network_minmax(len(w0))) * ncell,
            "network_ms": {"equal_weights": eq_ms, "unequal_weights": uneq_ms},
            "cells_with_p_above_half": int((exceed > 0.5).sum())}


def run_reference(args):
    world, rank, local = dist_setup(args)
    if rank != 0:
        return
    import oracle
    oracle.build()
    terr, hy, rm, sc, cells = make_inputs()
    p = oracle.Params(ny=NY, nx=NX)
    z = terr.z.astype(np.float64); n = terr.n.astype(np.float64)
    hy64 = hy.astype(np.float64)
    steps_per_sample = 2
    m = oracle.Member.dry(NY, NX, np.full((NY, NX), 0.05))
    for _ in range(args.warmup):
        oracle.advance(p, z, n, float(sc[0]), float(rm[0]), hy64, m, max_steps=steps_per_sample)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.advance(p, z, n, float(sc[0]), float(rm[0]), hy64, m, max_steps=steps_per_sample)
    el = time.perf_counter() - t0
    units = args.steps * steps_per_sample * NY * NX
    v = units / el
    sample = (f"each step: 1 member x {NY}x{NX} cells x {steps_per_sample} FP64 oracle steps "
              f"from a 5 cm wet start, 1 thread")
    print(json.dumps({
        "impl": "reference", "metric": "member-cell-steps/s", "value": v,
        "unit": "member-cell-steps/s", "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {**workload_config(), "parallelism": "replicas1",
                   "sample": "oracle, one member, two steps per benchmark step"},
        "cpu_baseline": {"value": v, "unit": "member-cell-steps/s", "cores": 1, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": v, "unit": "member-cell-steps/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0}}))


def run_gb300(args):
    import torch
    world, rank, local = dist_setup(args)
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    device = torch.device("cuda", local)
    torch.cuda.set_device(device)
    import __graft_entry__
    if rank == 0:
        __graft_entry__.build()
    barrier(world)
    from paper_2302_08341_gb300 import capi, synth
    capi.lib()

    terr, hy, rm, sc, cells = make_inputs()
    n_win = args.warmup + args.steps
    obs, truth = truth_observations(capi, terr, hy, cells, max(n_win, args.steps))
    stream = torch.cuda.current_stream(device)
    ncell = NY * NX

    g = capi.Grid(terr.z, terr.n)

    def window(gr, w, d_dev, beta_dev, u, outs):
        gr.advance_to(WINDOW * w, stream=stream)
        gr.gauge_sample(cells, out=outs["y"], stream=stream)
        gr.pf_assimilate(d_dev, 0.05, u, beta_dev, stream=stream, outputs=outs)

    # device-resident per-window inputs (observations, perturbations)
    d_all = [torch.tensor(o, dtype=torch.float64, device=device) for o in obs]
    draws = [synth.pf_draws(SEED, w, M) for w in range(1, max(n_win, args.steps) + 1)]
    beta_all = [torch.tensor(b, device=device) for _, b in draws]
    outs = dict(weights=torch.zeros(M, dtype=torch.float64, device=device),
                idx=torch.zeros(M, dtype=torch.int32, device=device),
                neff=torch.zeros(1, dtype=torch.float64, device=device),
                resampled=torch.zeros(1, dtype=torch.int32, device=device),
                y=torch.zeros((M, G), dtype=torch.float32, device=device))

    # warm-up windows, then the autotuner picks the step kernel's launch
    # configuration on the wet ensemble (and leaves it untouched)
    g.ensemble_init(M, rm, sc, hy, stream=stream)
    for w in range(1, args.warmup + 1):
        window(g, w, d_all[w - 1], beta_all[w - 1], draws[w - 1][0], outs)
    torch.cuda.synchronize(device)
    tuned = None
    if not args.no_autotune:
        rows_t, mpc_t, eng_t, ms_t = g.autotune(steps_per_trial=6, stream=stream)
        tuned = {"rows_per_strip": rows_t, "members_per_cta": mpc_t, "engine": eng_t,
                 "ms_per_step": ms_t}

    # timed windows from a fresh ensemble (the 1 h storm from t = 0)
    g.ensemble_init(M, rm, sc, hy, stream=stream)
    steps0 = g.members()["steps"].sum()
    launches0 = g.launch_count
    g.profile(True)
    start = torch.cuda.Event(enable_timing=True)
    stop = torch.cuda.Event(enable_timing=True)
    with Clocks(local) as clk:
        barrier(world)
        torch.cuda.synchronize(device)
        start.record(stream)
        for w in range(1, args.steps + 1):
            window(g, w, d_all[w - 1], beta_all[w - 1], draws[w - 1][0], outs)
        stop.record(stream)
        torch.cuda.synchronize(device)
        barrier(world)
    ms = start.elapsed_time(stop)
    kernel_ms, kernel_launches = g.profile(False)
    gpu_launches = g.launch_count - launches0
    units = float(g.members()["steps"].sum() - steps0) * ncell
    member_steps = units / ncell
    value, ms_max = job_value(units, ms, world, device)

    # roofline of the step kernel: algorithmic bytes / measured kernel time
    hbm_peak, peak_kind = peaks()
    achieved = member_steps * ncell * ALGO_BYTES / (kernel_ms * 1e-3) / 1e9
    tpu = traffic_per_unit()
    traffic = None if tpu is None else tpu * (member_steps / max(kernel_launches, 1)) * ncell
    roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                "frac": achieved / hbm_peak, "traffic": traffic,
                "kernel": "step_kernel", "peak_kind": peak_kind,
                "algorithmic_bytes_per_member_cell_step": ALGO_BYTES,
                "kernel_ms_total": kernel_ms, "kernel_launches": kernel_launches,
                "kernel_share_of_step": kernel_ms / ms if ms > 0 else None}

    # end to end through the public API with host buffers (pinned), copies
    # inside the timed region
    e2e = da_skill = None
    if not args.no_e2e:
        h_d = [torch.tensor(o, dtype=torch.float64).pin_memory() for o in obs]
        h_beta = [torch.tensor(b).pin_memory() for _, b in draws]
        h_outs = dict(weights=torch.zeros(M, dtype=torch.float64).pin_memory(),
                      idx=torch.zeros(M, dtype=torch.int32).pin_memory(),
                      neff=torch.zeros(1, dtype=torch.float64).pin_memory(),
                      resampled=torch.zeros(1, dtype=torch.int32).pin_memory(),
                      y=torch.zeros((M, G), dtype=torch.float32).pin_memory())
        g.ensemble_init(M, rm, sc, hy, stream=stream)
        g.set_graphs(True)   # runs of steps replayed from CUDA graphs (bit for bit the same)
        s0 = g.members()["steps"].sum()
        barrier(world)
        torch.cuda.synchronize(device)
        e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
        w_prior = np.full(M, 1.0 / M)   # the weights the members carry into a window
        est = []                        # per window: prior and posterior estimates at the gauges
        e0.record(stream)
        for w in range(1, args.steps + 1):
            window(g, w, h_d[w - 1], h_beta[w - 1], draws[w - 1][0], h_outs)
            stream.synchronize()   # the host reads the window's result
            _ = float(h_outs["neff"][0])
            y = h_outs["y"].numpy().astype(np.float64)
            w_post = h_outs["weights"].numpy().copy()
            est.append((w_prior @ y, w_post @ y))
            w_prior = np.full(M, 1.0 / M) if int(h_outs["resampled"][0]) else w_post
        e1.record(stream)
        torch.cuda.synchronize(device)
        barrier(world)
        g.set_graphs(False)
        e_ms = max_over_ranks(e0.elapsed_time(e1), world, device)
        e_units = sum_over_ranks(float(g.members()["steps"].sum() - s0) * ncell, world, device)
        e2e = {"value": e_units / (e_ms * 1e-3), "unit": "member-cell-steps/s",
               "h2d_bytes_per_step": G * 8 + M * 4,
               "d2h_bytes_per_step": M * 8 + M * 4 + 8 + 4 + M * G * 4}
        # what the filter does with the ensemble (§4.4): the weighted mean
        # depth at the gauges before and after each window's update, against
        # the hidden truth's own depths there
        pri = np.array([e[0] for e in est]); post = np.array([e[1] for e in est])
        tr = truth[:len(est)]
        da_skill = {"rmse_prior_m": float(np.sqrt(np.mean((pri - tr) ** 2))),
                    "rmse_posterior_m": float(np.sqrt(np.mean((post - tr) ** 2))),
                    "windows": len(est), "gauges": G,
                    "config": "weighted ensemble mean of the gauge depths before and after each "
                              "window's particle-filter update, against the hidden truth"}
    plain = products = eta = da = cfl = graphs = None
    if not args.no_extensions and world == 1:
        plain = plain_vs_fused(g, tuned, stream, device, ncell, hbm_peak)
        products = products_measure(g, stream, device, ncell, plain["fused"]["value"])
        eta = guarded(eta_sweeps, capi, g, tuned, stream, device, terr, hy, rm, sc)
        cfl = guarded(cfl_bound_measure, capi, terr, hy, rm, sc, tuned)
        graphs = guarded(graphs_measure, capi, terr, hy, rm, sc, tuned)
        da = guarded(assimilation_overhead, g, stream, device, cells, obs[0])
    g.close()
    extensions = {}
    if not args.no_extensions and world == 1:
        # a failing extension is reported on the line instead of losing it
        extensions["adjoint"] = guarded(adjoint_measure, capi)
        extensions["batched"] = guarded(batch_measure, capi, tune=True)
        pers = guarded(batch_measure, capi, engine=2,
                       rows=extensions["batched"].get("rows_per_strip"))
        if "error" not in extensions["batched"]:
            extensions["batched"]["hbm_frac_whole_window"] = (
                extensions["batched"]["value"] * BYTES_SINGLE / 1e9 / hbm_peak)
            extensions["batched"]["persistent"] = pers if "error" in pers else {
                **{k: pers[k] for k in ("value", "unit", "ms", "all_finished", "gpu_launches",
                                        "engine", "rows_per_strip")},
                "hbm_frac_whole_window": pers["value"] * BYTES_SINGLE / 1e9 / hbm_peak}
        bm = guarded(batch_measure, capi, tune=True, members=4)
        if "error" not in bm:
            # 24 B of state per member-cell-step, the bed and roughness once per tile of 4
            bm["hbm_frac_whole_window"] = bm["value"] * (BYTES_STATE + BYTES_STATIC / 4) / 1e9 / hbm_peak
        extensions["batched"]["four_members"] = bm
        bl = guarded(batch_measure, capi, tune=True, members=4, land_cover=True)
        if "error" not in bl:
            bl["hbm_frac_whole_window"] = (bl["active_value"] * (BYTES_STATE + BYTES_STATIC / 4)
                                           / 1e9 / hbm_peak)
        extensions["batched"]["land_cover"] = bl
        extensions["calibration"] = guarded(calibration_measure, capi,
                                            windows=args.calibration_windows)
        extensions["land_cover"] = guarded(land_cover_measure, capi)
        extensions["masked_domain"] = guarded(masked_domain_measure, capi)
        extensions["autotune"] = tuned
        extensions["plain_vs_fused"] = plain
        extensions["products"] = products
        extensions["eta_bar"] = eta
        extensions["cfl_bound"] = cfl
        extensions["graphs"] = graphs
        extensions["assimilation_overhead"] = da
        extensions["da_skill"] = da_skill

    if rank != 0:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        cpu = cpu_baseline(terr, hy, rm, sc)
        cpu["all_cores"] = cpu_all_cores(terr, hy, rm, sc)
    clocks = clk.summary()
    prod = extensions.get("products")
    if prod and "network_ops" in prod:
        # the product maps are bound by the ALU pipe (the sort network's
        # min/max), at the SM clock sampled during the timed windows
        mhz = (clocks or {}).get("sm_mhz") or 2070.0
        ops = prod.pop("network_ops")
        tms = prod.pop("network_ms")
        prod["alu_roofline"] = {k: alu_roofline(ops, v, mhz) for k, v in tms.items()}
    line = {
        "metric": "member-cell-steps/s", "value": value, "unit": "member-cell-steps/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {**workload_config(), "member_steps": member_steps,
                   "parallelism": f"replicas{world}",
                   "l2": "state 9.2 GB >> 129 MB L2 (no flush needed)"},
        "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": gpu_launches,
        "clocks": clocks,
    }
    line.update(rounded(extensions))
    if extensions:
        line["summary"] = extension_summary(extensions)
    print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_only(args):
    import torch
    torch.cuda.set_device(0)
    import __graft_entry__
    __graft_entry__.build()
    from paper_2302_08341_gb300 import capi
    capi.lib()
    if args.only == "adjoint":
        res = adjoint_measure(capi)
    elif args.only == "batch":
        res = batch_measure(capi, engine=args.engine, tune=args.engine is None and not ROWS)
    elif args.only == "batch_land_cover":
        res = batch_measure(capi, engine=args.engine, tune=args.engine is None and not ROWS,
                            members=4, land_cover=True)
    elif args.only == "land_cover":
        res = land_cover_measure(capi)
    elif args.only == "masked_domain":
        res = masked_domain_measure(capi)
    elif args.only == "products":
        res = products_only(capi)
    else:
        res = calibration_measure(capi, windows=args.calibration_windows)
    print(json.dumps({"only": args.only, "members": M, "cells": NY * NX, **res}))


def main():
    args = parse()
    if args.only:
        run_only(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gb300(args)


if __name__ == "__main__":
    main()
