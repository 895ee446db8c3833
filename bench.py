#!/usr/bin/env python
"""Throughput of the tree gravity + tree collision step on GB300.

Workload: the 1,000,000-particle shearing sheet (box 2050 x 2050 m, R = 1 m,
rho = 400 kg/m^3, z ~ N(0, 1 m), shear flow plus dispersion 2 Omega x 1 m),
1 ghost ring in x and y, open z, SEI, Barnes-Hut theta = 0.5 with quadrupoles,
FP32 cell-relative walk, hard-sphere collisions with eps = 0.5.  A step is one
full DKD step (drift, tree build, gravity walk, kick, drift, collision tree,
collision search, pair sort, resolution).  Metric: particle-steps/s.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank advances its own independent sheet on its own GPU
(replicas; weak scaling) and rank 0 prints one JSON line.  --impl reference
times the FP64 CPU oracle (the only reference this method has) on the host
cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "particle-steps/s (tree gravity+collisions, N=1M) at fixed force error vs direct sum"
UNIT = "particle-steps/s"
N_SHEET = 1_000_000
L_SHEET = 2050.0
SEED = 5
FP32_LANES_PER_SM = 128
# algorithmic bytes per particle of one tree build (sort + gather, topology,
# moments): each 8-bit radix pass reads and writes an 8-byte key and a 4-byte
# value; the gather reads and writes the 64-byte FP64 state plus id and box
# (8 B) and writes the slot of each id (4 B); the topology reads each key
# once; each tree cell writes ~160 B of FP64 and FP32 records
BUILD_PASSES = 8
BYTES_PASS, BYTES_GATHER, BYTES_KEYS, BYTES_CELL = 24, 148, 8, 160
BYTES_DIGITS = 8   # one read of the keys counts the digits of every pass
# algorithmic FP32 flops per interaction (FMA = 2, add/mul = 1, rsqrt = 0)
FLOP_CELL, FLOP_LEAF, FLOP_MAC = 60, 20, 10
FLOP_MLP = 2 * (12 * 64 + 2 * 64 * 64 + 64 * 3)


def workload_name(walk: str) -> str:
    tree = ("theta=0.8 quadrupole + learned residual for w/R > 0.5 (BF16 MLP)" if walk == "learned"
            else f"theta=0.5 quadrupole, {walk} walk")
    return (f"shearing sheet N={N_SHEET:,} box {L_SHEET:g}x{L_SHEET:g} m, 1 ghost ring, SEI, "
            f"{tree}, collisions eps=0.5")


def sheet_config(rb, walk):
    from paper_1110_4876_gb300 import inputs as I

    mode = {"fp32": rb.RB_WALK_FP32, "fp64": rb.RB_WALK_FP64, "learned": rb.RB_WALK_FP32_LEARNED}[walk]
    return dict(G=I.G_SI, omega=I.OMEGA, box=(L_SHEET,) * 3, nghost=(1, 1, 0),
                boundary=rb.RB_BC_SHEAR, integrator=rb.RB_INT_SEI,
                theta=0.8 if walk == "learned" else 0.5, eps=0.5, dt=I.DT_SHEET, gravity=1,
                collisions=1, walk=mode)


_WEIGHTS = {}


def make_sim(rb, cfg, stream=None, nbox=1):
    """A simulation; in the learned mode the network is trained once per
    process (librb's own kernels) and loaded."""
    sim = rb.Sim(nbox=nbox, stream=stream, **cfg)
    if cfg["walk"] == rb.RB_WALK_FP32_LEARNED:
        if "w" not in _WEIGHTS:
            from paper_1110_4876_gb300 import learned

            _WEIGHTS["w"], _WEIGHTS["loss"] = learned.train_default()
        rb.rb_load_mlp(sim.h, _WEIGHTS["w"], 0.5)
    return sim


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


class Clocks:
    """nvidia-smi sampling (every 20 ms, timestamped) of SM clocks and throttle
    reasons.  The sampler starts before the warm-up, so it is running when the
    timed window opens; window(t0, t1) marks that window in host time and
    summary() keeps the samples taken inside it."""

    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.path = None
        self.t0 = self.t1 = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "20"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def window(self, t0: float, t1: float):
        self.t0, self.t1 = t0, t1

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    @staticmethod
    def _epoch(stamp: str):
        import datetime

        for fmt in ("%Y/%m/%d %H:%M:%S.%f", "%Y/%m/%d %H:%M:%S"):
            try:
                return datetime.datetime.strptime(stamp, fmt).timestamp()
            except ValueError:
                pass
        return None

    def summary(self):
        if not self.proc or not self.path:
            return None
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 10:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        inside = rows
        if self.t0 is not None:
            inside = [r for r in rows if (t := self._epoch(r[0])) is not None and self.t0 <= t <= self.t1]
        use = inside if inside else rows
        sm = [float(r[2]) for r in use if r[2].replace(".", "").isdigit()]
        mx = [float(r[3]) for r in use if r[3].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in use for k in range(4) if r[6 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(inside), "samples_whole_run": len(rows),
                "window_s": (self.t1 - self.t0) if self.t0 is not None else None}


def max_over_ranks(t_ms: float, dist, device) -> float:
    """The slowest rank's time (all ranks call this)."""
    if not dist:
        return t_ms
    import torch

    t = torch.tensor([t_ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def search_rate(visits, iters, ms, ms_counted):
    """Tree collision search: tree entries tested by the targets (nodes
    visited, all images) per launch, counted by the search's counting
    variant in one step after the timed ones, over the event-timed search
    stage of the timed steps (which run the plain variant).  The search is
    bound by L1/L2 latency, so it is reported as a rate, with no roofline."""
    if not (visits > 0 and ms > 0):
        return None
    return {"bound": "latency (L1/L2 round trips)", "kernel": "k_collide (tree collision search)",
            "nodes_visited_per_launch": visits, "nodes_visited_per_particle": visits / N_SHEET,
            "nodes_visited_per_s": visits / (ms / 1e3), "ms_per_launch": ms,
            "warp_iterations_per_launch": iters,
            "lane_utilisation": visits / (32.0 * iters) if iters > 0 else None,
            "counted": "in one step after the timed steps, by the counting variant "
                       f"({ms_counted:.4f} ms); the timed steps run the plain search"}


def whole_job_value(world: int, n_per_rank: int, steps: int, t_ms: float) -> float:
    """Particle-steps/s of all ranks together (each rank advances its own
    n_per_rank particles for `steps` steps; t_ms is the slowest rank)."""
    return world * n_per_rank * steps / (t_ms / 1e3)


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def run_ours(args):
    import torch

    from paper_1110_4876_gb300 import inputs as I
    from paper_1110_4876_gb300 import rb

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    rb.load()
    stream = torch.cuda.Stream()
    cfg = sheet_config(rb, args.walk)
    P = I.sheet(L_SHEET, N_SHEET, SEED + rank)
    sim = make_sim(rb, cfg, stream.cuda_stream)
    sim.set_particles(P)
    if args.shape:
        rb.rb_set_launch_shape(sim.h, *args.shape)
        tuned = tuple(args.shape)
    else:
        tuned = rb.rb_autotune(sim.h)
    rb.rb_set_profiling(sim.h, True)
    clk = Clocks(local).__enter__()   # sampling from before the warm-up
    sim.step(args.warmup)

    def barrier():
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()

    # ---- device-resident throughput (inputs already in HBM) ----
    walk_ms, walk_flops, stage_sum = [], [], {}
    launches = 0
    pairs, corr, counts, cells, search_ms = [], [], [], [], []
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    barrier()
    tw0 = time.time()
    e0.record(stream)
    for _ in range(args.steps):
        sim.step(1)
        st = sim.stats()
        walk_ms.append(st["ms_stage"]["gravity_walk"])
        walk_flops.append(FLOP_CELL * st["cell_interactions"] + FLOP_LEAF * st["leaf_interactions"]
                          + FLOP_MAC * st["mac_tests"])
        for k, v in st["ms_stage"].items():
            stage_sum[k] = stage_sum.get(k, 0.0) + v
        launches += st["kernels_per_step"]
        pairs.append(st["pairs_found"])
        corr.append(st["corrections"])
        counts.append((st["cell_interactions"], st["leaf_interactions"], st["mac_tests"],
                       st["warp_iterations"]))
        cells.append(st["cells"])
        search_ms.append(st["ms_stage"]["collision_search"])
    e1.record(stream)
    barrier()
    clk.window(tw0, time.time())
    clk.__exit__()
    t_ms = max_over_ranks(e0.elapsed_time(e1), dist, "cuda")
    clocks = clk.summary()
    value = whole_job_value(world, N_SHEET, args.steps, t_ms)
    # one more step, untimed, with the counting variant of the collision search
    rb.rb_set_profiling(sim.h, 2)
    sim.step(1)
    st = sim.stats()
    search = search_rate(st["search_visits"], st["search_iterations"],
                         statistics.mean(search_ms), st["ms_stage"]["collision_search"])
    rb.rb_set_profiling(sim.h, 1)

    # ---- end to end through the C ABI with host buffers ----
    ke = max(3, min(args.steps, 10))
    fields = ("x", "y", "z", "vx", "vy", "vz", "m", "r")

    def pinned():
        return {k: torch.empty(N_SHEET, dtype=torch.float64).pin_memory().numpy() for k in fields}

    bufs = [pinned(), pinned()]
    for k, a in zip(fields, P.arrays()):
        bufs[0][k][:] = a
    sim_e = make_sim(rb, cfg, stream.cuda_stream)
    sim_e.set_particles(tuple(bufs[0][k] for k in fields))
    rb.rb_set_launch_shape(sim_e.h, *tuned)   # the launch shapes chosen above
    sim_e.step(1)  # capture the step graphs outside the timed region
    sim_e.particles(out=bufs[1])
    barrier()
    t0 = time.perf_counter()
    for k in range(ke):
        src, dst = bufs[k & 1], bufs[(k + 1) & 1]
        sim_e.set_particles(tuple(src[f] for f in fields))   # host -> device
        sim_e.step(1)
        sim_e.particles(out=dst)                                # device -> host
    barrier()
    te = time.perf_counter() - t0
    e2e = {"value": world * N_SHEET * ke / te, "unit": UNIT,
           "h2d_bytes_per_step": 8 * 8 * N_SHEET, "d2h_bytes_per_step": 8 * 8 * N_SHEET,
           "steps": ke, "host_buffers": "pinned, reused; each step copies the previous step's "
                                        "output back in"}
    del sim_e

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return None

    peaks = measured_peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    fp32_peak = sms * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
    wms = statistics.mean(walk_ms)
    if not wms > 0.0:
        raise RuntimeError("the gravity walk stage time was not recorded")
    achieved = statistics.mean(walk_flops) / (wms / 1e3) / 1e12
    kname = ("k_walk32_learn (gravity walk with the in-walk MLP; FP32 flops only)"
             if args.walk == "learned" else "k_walk32 (gravity walk)")
    traffic, traffic_note = profiled_traffic("gravity_walk_sheet1m.md", WALK_SOURCES)
    roofline = {"bound": "alu", "kernel": kname, "achieved": achieved,
                "peak": fp32_peak, "unit": "TFLOP/s", "frac": achieved / fp32_peak,
                "traffic": traffic, "traffic_source": traffic_note, "peak_source":
                    f"derived: {sms} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 x {sm_max:g} MHz "
                    "(MEASURED_PEAKS.json sm_max_mhz; the device's SM count)",
                "flops_per_launch": statistics.mean(walk_flops), "ms_per_launch": wms}
    ncell, nleaf, nmac, niter = (statistics.mean(c[k] for c in counts) for k in range(4))
    roofline["per_particle"] = {"cells": ncell / N_SHEET, "leaves": nleaf / N_SHEET,
                                "opening_tests": nmac / N_SHEET}
    if niter > 0:
        # entries a lane evaluates / entries the warps step through x 32 lanes
        roofline["warp_iterations_per_launch"] = niter
        roofline["lane_utilisation"] = (nleaf + nmac) / (32.0 * niter)
    if args.walk == "learned":
        # tensor-core work of the network: 2 (12 64 + 2 64 64 + 64 3) flops per corrected cell
        mlp = FLOP_MLP * statistics.mean(corr)
        roofline["mlp"] = {"corrections_per_launch": statistics.mean(corr), "flops_per_launch": mlp,
                           "tflops": mlp / (wms / 1e3) / 1e12, "path": "mma.sync m16n8k16 BF16"}
        roofline["traffic"] = None
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64" if args.walk == "fp64" else "f32",
        "data": "synthetic (seeded shearing-sheet generator; no dataset or weights)",
        "config": {"workload": workload_name(args.walk), "particles_per_gpu": N_SHEET,
                   "parallelism": "replicas" if world > 1 else "single",
                   "precision": ("all FP64" if args.walk == "fp64" else
                                 "walk FP32 on hi/lo cell-relative offsets; positions, kick/drift, "
                                 "moments, collisions FP64" +
                                 ("; MLP BF16 weights, FP32 accumulate" if args.walk == "learned"
                                  else "")),
                   "l2": "no flush: working set (2 x 72 MB particle sets + ~0.4 GB tree) > 129 MB L2",
                   "pairs_per_step": statistics.mean(pairs),
                   "walk_block, search_block, walk_group, tile_order": list(tuned)},
        "clocks": clocks, "e2e": e2e, "gpu_launches": launches, "roofline": roofline,
        "roofline_build": build_roofline(stage_sum, args.steps, cells, peaks, tuned[3]),
        "collision_search": search,
        "stage_ms_per_step": {k: v / args.steps for k, v in stage_sum.items()},
    }
    if args.cpu_baseline and world == 1:
        line["cpu_baseline"], line["force_error"] = cpu_baseline(sim, cfg, P, args)
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return line


WALK_SOURCES = ("paper_1110_4876_gb300/csrc/rb_walk.cu", "paper_1110_4876_gb300/csrc/rb_internal.cuh")
BUILD_SOURCES = ("paper_1110_4876_gb300/csrc/rb_sort.cu", "paper_1110_4876_gb300/csrc/rb_step.cu",
                 "paper_1110_4876_gb300/csrc/rb_tree.cu", "paper_1110_4876_gb300/csrc/rb_internal.cuh")


def source_hash(paths) -> str:
    """sha256 over the kernel sources (the build that a capture measured)."""
    import hashlib

    h = hashlib.sha256()
    for rel in paths:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def profiled_traffic(summary: str, sources, field: str = "dram_bytes_per_launch"):
    """DRAM bytes (per launch, or per build) of the 1M sheet from a committed
    ncu summary, if it was taken on the current kernel sources (its
    `source_sha256:` line equals the hash of `sources`) and the run is that
    workload; else None.  Returns (bytes or None, note)."""
    if (N_SHEET, L_SHEET) != (1_000_000, 2050.0):
        return None, f"profiles/{summary} holds the 1M sheet's traffic; this run is another workload: null"
    path = os.path.join(ROOT, "profiles", summary)
    fields = {}
    try:
        with open(path) as f:
            for line in f:
                if ":" in line and line.split(":", 1)[0] in (field, "source_sha256"):
                    k, v = line.split(":", 1)
                    fields[k] = v.strip()
    except OSError:
        return None, f"no capture summary profiles/{summary}"
    now = source_hash(sources)
    if fields.get("source_sha256") != now or field not in fields:
        return None, f"profiles/{summary} was taken on other kernel sources (now {now}): null"
    return float(fields[field]), f"ncu capture in profiles/{summary} (sources {now})"


def build_roofline(stage_sum, steps, cells, peaks, tile_order=0):
    """HBM roofline of the tree build (sort + gather, topology, tile order,
    moments) from the event-timed stages: algorithmic bytes per step / stage
    time."""
    n = N_SHEET
    ncells = statistics.mean(cells) if cells else 0.0
    per_particle = BYTES_DIGITS + BUILD_PASSES * BYTES_PASS + BYTES_GATHER + BYTES_KEYS
    if tile_order:
        # Hilbert tile keys: read the Morton key (8 B), write key and slot
        # (12 B), then the digit counts and 3 radix passes of 24 B
        per_particle += 20 + BYTES_DIGITS + 3 * BYTES_PASS
    nbytes = n * per_particle + ncells * BYTES_CELL
    ms = sum(stage_sum.get(k, 0.0) for k in ("sort_gather", "tree", "moments")) / steps
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    achieved = nbytes / (ms / 1e3) / 1e9 if ms > 0 else None
    traffic, note = profiled_traffic("tree_build_sheet1m.md", BUILD_SOURCES, "dram_bytes_per_build")
    return {"bound": "hbm", "kernels": "k_rs_hist + k_rs_pass (8 passes), k_permute, topology, "
                                       "tile order (k_tile_keys, k_rs_hist + 3 passes), k_moments_level (per depth)",
            "achieved": achieved, "peak": hbm, "unit": "GB/s",
            "frac": achieved / hbm if achieved else None, "traffic": traffic, "traffic_source": note,
            "bytes_per_step": nbytes, "ms_per_step": ms, "cells_per_particle": ncells / n,
            "bytes_model": f"digit counts {BYTES_DIGITS} B + {BUILD_PASSES} radix passes x {BYTES_PASS} B + "
                           f"gather {BYTES_GATHER} B + keys {BYTES_KEYS} B per particle + {BYTES_CELL} B per cell"
                           + (" + tile order 100 B per particle" if tile_order else ""),
            "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured copy bandwidth)"}


def oracle_sample(P, samples: int, seed: int = 0):
    """Time the oracle's step on the workload: drifts and tree builds on all
    N particles, the gravity walk and the collision search from a random
    sample of targets, scaled per particle; returns (seconds per
    particle-step, details, threads, params, sample)."""
    import oracle
    from paper_1110_4876_gb300 import inputs as I

    p = oracle.Params(G=I.G_SI, omega=I.OMEGA, L=(L_SHEET,) * 3, nghost=(1, 1, 0), boundary=2,
                      integrator=1, theta=0.5, eps=0.5, dt=I.DT_SHEET, gravity=1, collisions=1)
    n = P.n
    t = time.perf_counter()
    s = oracle.drift(p, P.x, P.y, P.z, P.vx, P.vy, P.vz)
    t_drift = time.perf_counter() - t
    t = time.perf_counter()
    tree = oracle.Tree(s[0], s[1], s[2], P.m, L_SHEET)
    t_build = time.perf_counter() - t
    sel = np.random.default_rng(seed).choice(n, samples, replace=False)
    t = time.perf_counter()
    tree.gravity(p, oracle.time_at(p, 1), targets=sel)
    t_walk = time.perf_counter() - t
    # the collision search from the sampled targets, timed on its own (Eq. 3
    # reads only the cells' geometry, so this tree serves; the step's second
    # build is counted above)
    t = time.perf_counter()
    keys = tree.collide(p, oracle.time_at(p, 2), P.r, np.arange(n), sel)
    t_search = time.perf_counter() - t
    del tree
    per = (2 * t_drift + 2 * t_build) / n + (t_walk + t_search) / samples
    detail = (f"N={n:,}: drift x2 {2 * t_drift:.2f} s and two tree builds {2 * t_build:.2f} s on "
              f"all particles; gravity walk {t_walk:.2f} s and collision search "
              f"{t_search:.2f} s ({len(keys)} pairs) from {samples} random targets, scaled per "
              f"particle; resolution not timed (under 1% of the oracle step)")
    return per, detail, oracle.nthreads(), p, sel


def oracle_full_step(P):
    """One whole oracle step of the workload on the host cores: drift, tree
    build, gravity walk of every particle over the ghost images, kick, drift,
    collision tree search and resolution.  Returns (seconds, pairs, threads)."""
    import oracle
    from paper_1110_4876_gb300 import inputs as I

    p = oracle.Params(G=I.G_SI, omega=I.OMEGA, L=(L_SHEET,) * 3, nghost=(1, 1, 0), boundary=2,
                      integrator=1, theta=0.5, eps=0.5, dt=I.DT_SHEET, gravity=1, collisions=1)
    st = oracle.State(p, *P.arrays())
    t = time.perf_counter()
    st.step(1)
    return time.perf_counter() - t, len(st.last_pairs), oracle.nthreads()


def cpu_baseline(sim, cfg, P, args):
    """The oracle on this host's cores (one whole step of the workload) and
    the force error of the GPU walk against the oracle's direct sum and its
    tree at the same theta on 4096 seeded targets."""
    import oracle
    from paper_1110_4876_gb300 import inputs as I
    from paper_1110_4876_gb300 import rb

    secs, npairs, cores = oracle_full_step(P)
    base = {"value": P.n / secs, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"one whole oracle step of the N={P.n:,} sheet ({secs:.1f} s on {cores} threads): "
                      f"drift, tree build, gravity walk of every particle over 9 images, kick, drift, "
                      f"tree collision search ({npairs} pairs), resolution"}
    p = oracle.Params(G=I.G_SI, omega=I.OMEGA, L=(L_SHEET,) * 3, nghost=(1, 1, 0), boundary=2,
                      integrator=1, theta=0.5, eps=0.5, dt=I.DT_SHEET, gravity=1, collisions=1)
    # force error of the benchmarked walk at the initial state
    sim_f = make_sim(rb, cfg)
    sim_f.set_particles(P)
    a_gpu = sim_f.gravity()
    sel = np.random.default_rng(1).choice(P.n, 4096, replace=False)
    a_dir = oracle.direct_gravity(p, 0.0, P.x, P.y, P.z, P.m, targets=sel)
    a_tree = oracle.Tree(P.x, P.y, P.z, P.m, L_SHEET).gravity(p, 0.0, targets=sel)
    es, rr, mr = oracle.force_errors(a_gpu[sel], a_dir)
    _, _, mt = oracle.force_errors(a_gpu[sel], a_tree)
    fe = {"vs_direct_sum": {"e_sum": es, "rms_rel": rr, "max_rel": mr},
          "vs_oracle_tree_same_theta": {"max_rel": mt}, "targets": 4096,
          "floor": "per-particle denominator floored at 1e-3 rms|a|"}
    return base, fe


def run_ensemble(args):
    """256 shearing boxes of uneven N advanced together (every stage one
    launch over all boxes, one CUDA graph per step) against the same boxes as
    256 single-box simulations stepped one after another.  Prints one JSON
    line (not the headline metric)."""
    import torch

    from paper_1110_4876_gb300 import inputs as I
    from paper_1110_4876_gb300 import rb

    rb.load()
    stream = torch.cuda.Stream()
    boxes = I.ensemble_boxes(256)
    parts = [(Lb, I.sheet(Lb, nb, seed + 7919)) for nb, Lb, seed in boxes]
    ntot = sum(P.n for _, P in parts)

    def cfg(L):
        c = sheet_config(rb, args.walk)
        c["box"] = (L, L, L)
        return c

    ens = rb.Sim(nbox=len(parts), stream=stream.cuda_stream, **cfg(parts[0][0]))
    for b, (Lb, P) in enumerate(parts):
        ens.set_box(b, (Lb, Lb, Lb))
        ens.set_particles(P, box=b)
    if args.shape:
        rb.rb_set_launch_shape(ens.h, *args.shape)   # fixed shapes (profiling runs)
        tuned = tuple(args.shape)
    else:
        tuned = rb.rb_autotune(ens.h)
    clk = Clocks(torch.cuda.current_device()).__enter__()
    ens.step(args.warmup)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    tw0 = time.time()
    e0.record(stream)
    ens.step(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    clk.window(tw0, time.time())
    clk.__exit__()
    t_batched = e0.elapsed_time(e1) / 1e3
    # per-stage split of the batched step, from a separate profiled pass
    rb.rb_set_profiling(ens.h, True)
    stage_sum, pairs = {}, 0
    for _ in range(args.steps):
        ens.step(1)
        st = ens.stats()
        pairs += st["pairs_found"]
        for k, v in st["ms_stage"].items():
            stage_sum[k] = stage_sum.get(k, 0.0) + v
    rb.rb_set_profiling(ens.h, False)
    singles = []
    for Lb, P in parts:
        s = rb.Sim(stream=stream.cuda_stream, **cfg(Lb))
        s.set_particles(P)
        s.step(1)
        singles.append(s)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        for s in singles:
            s.step(1)
    e1.record(stream)
    torch.cuda.synchronize()
    t_looped = e0.elapsed_time(e1) / 1e3
    line = {"metric": "particle-steps/s (256-box shearing-sheet ensemble)", "unit": UNIT,
            "value": ntot * args.steps / t_batched, "looped_single_boxes": ntot * args.steps / t_looped,
            "speedup": t_looped / t_batched, "particles": ntot, "boxes": len(parts),
            "steps": args.steps, "warmup": args.warmup, "walk_block, search_block, walk_group, tile_order": list(tuned),
            "pairs_per_step": pairs / args.steps,
            "stage_ms_per_step (profiled pass)": {k: v / args.steps for k, v in stage_sum.items()},
            "clocks (batched timed region)": clk.summary(),
            "dtype": "f64" if args.walk == "fp64" else "f32", "data": "synthetic",
            "config": {"workload": "256 shearing boxes, N_b log-uniform [500, 20000], surface "
                                   "density log-uniform [200, 1000] kg/m^2, theta=0.5, SEI, eps=0.5"}}
    print(json.dumps(line), flush=True)
    return line


def _timed(sim, stream, steps, warmup):
    """ms per step (CUDA events on the library's stream), the gravity walk
    stage's ms per step, after warm-up and autotuning, and the launch shape
    the autotuner chose (walk block, search block, walk group, tile order)."""
    import torch

    from paper_1110_4876_gb300 import rb

    shape = rb.rb_autotune(sim.h)
    rb.rb_set_profiling(sim.h, True)
    sim.step(warmup)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    walk = 0.0
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(steps):
        sim.step(1)
        walk += sim.stats()["ms_stage"]["gravity_walk"]
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps, walk / steps, list(shape)


def _errors(a, a_ref):
    import oracle

    es, rr, mr = oracle.force_errors(a, a_ref)
    return {"e_sum": es, "rms_rel": rr, "max_rel": mr}


def run_compare(args):
    """The 1M sheet's step with each walk form (FP64 and FP32 at theta 0.5,
    plain FP32 and learned at theta 0.8): particle-steps/s next to the force
    error against the oracle's direct sum on 4096 seeded targets (all ghost
    images).  One JSON line."""
    import torch

    import oracle
    from paper_1110_4876_gb300 import inputs as I
    from paper_1110_4876_gb300 import rb

    rb.load()
    stream = torch.cuda.Stream()
    clk = Clocks(torch.cuda.current_device()).__enter__()
    t_clk = time.time()
    P = I.sheet(L_SHEET, N_SHEET, SEED)
    sel = np.random.default_rng(1).choice(P.n, 4096, replace=False)
    p = oracle.Params(G=I.G_SI, omega=I.OMEGA, L=(L_SHEET,) * 3, nghost=(1, 1, 0), boundary=2,
                      integrator=1, theta=0.5, eps=0.5, dt=I.DT_SHEET, gravity=1, collisions=1)
    t = time.perf_counter()
    a_dir = oracle.direct_gravity(p, 0.0, P.x, P.y, P.z, P.m, targets=sel)
    t_dir = time.perf_counter() - t
    rows = {}
    for name, walk, theta in [("fp64 theta=0.5", "fp64", 0.5), ("fp32 theta=0.5", "fp32", 0.5),
                              ("fp32 theta=0.8", "fp32", 0.8), ("learned theta=0.8", "learned", 0.8)]:
        cfg = sheet_config(rb, walk)
        cfg["theta"] = theta
        sim = make_sim(rb, cfg, stream.cuda_stream)
        sim.set_particles(P)
        a = sim.gravity()
        err = _errors(a[sel], a_dir)
        sim.set_particles(P)
        ms, wms, shape = _timed(sim, stream, args.steps, args.warmup)
        rows[name] = {"particle_steps_per_s": N_SHEET / (ms / 1e3), "ms_per_step": ms,
                      "walk_ms": wms, "force_error_vs_direct": err, "launch_shape": shape}
        del sim
    clk.window(t_clk, time.time())
    clk.__exit__()
    line = {"metric": "particle-steps/s and force error vs direct sum per walk form (1M sheet)",
            "unit": UNIT, "steps": args.steps, "warmup": args.warmup, "forms": rows,
            "direct_sum": {"targets": 4096, "images": 9, "seconds": t_dir, "cores": oracle.nthreads()},
            "data": "synthetic", "config": {"workload": workload_name("fp32")}}
    line["clocks (whole run)"] = clk.summary()
    print(json.dumps(line), flush=True)
    return line


def run_extensions(args):
    """The 1M sheet's step (FP32 walk, theta 0.5) with the velocity-dependent
    restitution and the test particles the paper allows (Sect. 5 and
    Sect. 4): the constant eps = 0.5 as in the default run, an illustrative
    power law eps = min(1, (|v_n| / v_c)^-p) with v_c = 7.7e-5 m/s and
    p = 0.234 (about 0.75 at the sheet's impact speeds), and the ids above
    N/2 as test particles.  Their parity with the oracle is tested in
    tests/test_gpu_extensions.py.  One JSON line."""
    import torch

    from paper_1110_4876_gb300 import inputs as I
    from paper_1110_4876_gb300 import rb

    rb.load()
    stream = torch.cuda.Stream()
    clk = Clocks(torch.cuda.current_device()).__enter__()
    t_clk = time.time()
    P = I.sheet(L_SHEET, N_SHEET, SEED)
    rows = {}
    for name in ("constant eps=0.5", "power-law eps (v_c=7.7e-5 m/s, p=0.234)", "test particles (n_active=N/2)"):
        sim = make_sim(rb, sheet_config(rb, "fp32"), stream.cuda_stream)
        if name.startswith("power"):
            rb.rb_set_restitution(sim.h, rb.RB_EPS_POWER, 7.7e-5, 0.234)
        if name.startswith("test"):
            rb.rb_set_n_active(sim.h, N_SHEET // 2)
        sim.set_particles(P)
        ms, wms, shape = _timed(sim, stream, args.steps, args.warmup)
        st = sim.stats()
        rows[name] = {"particle_steps_per_s": N_SHEET / (ms / 1e3), "ms_per_step": ms, "walk_ms": wms,
                      "pairs_last_step": st["pairs_found"], "launch_shape": shape}
        del sim
    clk.window(t_clk, time.time())
    clk.__exit__()
    line = {"metric": "particle-steps/s with the restitution law and test particles (1M sheet)",
            "unit": UNIT, "steps": args.steps, "warmup": args.warmup, "forms": rows,
            "data": "synthetic", "config": {"workload": workload_name("fp32")}}
    line["clocks (whole run)"] = clk.summary()
    print(json.dumps(line), flush=True)
    return line


def run_plummer(args):
    """Plummer sphere, N = 2^20 (G = M = a = 1, open, leap-frog, dt = 1e-3,
    softening 1e-3): the FP32 and FP64 walks at theta 0.3 / 0.5 / 0.7,
    particle-steps/s and force error against the oracle's direct sum on 4096
    seeded targets.  One JSON line."""
    import torch

    import oracle
    from paper_1110_4876_gb300 import inputs as I
    from paper_1110_4876_gb300 import rb

    rb.load()
    stream = torch.cuda.Stream()
    clk = Clocks(torch.cuda.current_device()).__enter__()
    t_clk = time.time()
    n = 1 << 20
    P = I.plummer(n, 3)
    sel = np.random.default_rng(1).choice(P.n, 4096, replace=False)
    p = oracle.Params(G=1.0, L=(128.0,) * 3, theta=0.5, soft=1e-3, dt=1e-3, gravity=1)
    t = time.perf_counter()
    a_dir = oracle.direct_gravity(p, 0.0, P.x, P.y, P.z, P.m, targets=sel)
    t_dir = time.perf_counter() - t
    rows = {}
    for theta in (0.3, 0.5, 0.7):
        for walk, mode in (("fp32", rb.RB_WALK_FP32), ("fp64", rb.RB_WALK_FP64)):
            cfg = dict(G=1.0, box=(128.0,) * 3, boundary=rb.RB_BC_OPEN, integrator=rb.RB_INT_LEAPFROG,
                       theta=theta, softening=1e-3, dt=1e-3, gravity=1, collisions=0, walk=mode)
            sim = rb.Sim(stream=stream.cuda_stream, **cfg)
            sim.set_particles(P)
            a = sim.gravity()
            err = _errors(a[sel], a_dir)
            sim.set_particles(P)
            ms, wms, shape = _timed(sim, stream, args.steps, args.warmup)
            rows[f"{walk} theta={theta}"] = {"particle_steps_per_s": n / (ms / 1e3), "ms_per_step": ms,
                                             "walk_ms": wms, "force_error_vs_direct": err,
                                             "launch_shape": shape}
            del sim
    clk.window(t_clk, time.time())
    clk.__exit__()
    line = {"metric": "particle-steps/s and force error vs direct sum, Plummer N=2^20", "unit": UNIT,
            "steps": args.steps, "warmup": args.warmup, "forms": rows,
            "direct_sum": {"targets": 4096, "seconds": t_dir, "cores": oracle.nthreads()},
            "data": "synthetic (seeded Plummer sampler)",
            "config": {"workload": "Plummer G=M=a=1, N=1,048,576, open box 128, leap-frog dt=1e-3, "
                                   "softening 1e-3, quadrupole, no collisions"}}
    line["clocks (whole run)"] = clk.summary()
    print(json.dumps(line), flush=True)
    return line


def run_sweep(args):
    """Collision detectors on non-self-gravitating shearing sheets (the
    paper's collision scaling test, Sect. 7): the plane sweep (Sect. 5.3) and
    the tree search (Sect. 5.2) on an elongated box (azimuthal size 20 R,
    optical depth 0.75) and on the square 1M sheet.  Whole collision-only
    steps (drift, detection, pair sort, resolution), particle-steps/s, and the
    detection's share.  One JSON line."""
    import torch

    from paper_1110_4876_gb300 import inputs as I
    from paper_1110_4876_gb300 import rb

    rb.load()
    stream = torch.cuda.Stream()
    clk = Clocks(torch.cuda.current_device()).__enter__()
    t_clk = time.time()
    rows = {}
    n = args.particles
    Ly = 20.0
    Lx = I.long_sheet_size(n, Ly)
    cases = [("elongated", Lx, Ly, lambda: I.sheet_xy(Lx, Ly, n, SEED)),
             ("square", L_SHEET, L_SHEET, lambda: I.sheet(L_SHEET, N_SHEET, SEED))]
    for name, lx, ly, make in cases:
        if name not in args.cases.split(","):
            continue
        P = make()
        for det, code in (("sweep", rb.RB_COLL_SWEEP), ("tree", rb.RB_COLL_TREE)):
            cfg = dict(G=I.G_SI, omega=I.OMEGA, box=(lx, ly, lx), nghost=(1, 1, 0),
                       boundary=rb.RB_BC_SHEAR, integrator=rb.RB_INT_SEI, eps=0.5, dt=I.DT_SHEET,
                       gravity=0, collisions=code)
            sim = rb.Sim(stream=stream.cuda_stream, **cfg)
            sim.set_particles(P)
            try:
                rb.rb_autotune(sim.h)
                rb.rb_set_profiling(sim.h, True)
                sim.step(args.warmup)
            except rb.RbError as e:
                rows[f"{name} {det}"] = {"error": str(e)}
                continue
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            st_sum = {}
            pairs = 0
            torch.cuda.synchronize()
            e0.record(stream)
            for _ in range(args.steps):
                sim.step(1)
                st = sim.stats()
                pairs += st["pairs_found"]
                for k, v in st["ms_stage"].items():
                    st_sum[k] = st_sum.get(k, 0.0) + v
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / args.steps
            det_ms = sum(st_sum.get(k, 0.0) for k in ("sort_gather_c", "tree_c", "collision_records",
                                                      "collision_search")) / args.steps
            rows[f"{name} {det}"] = {"particles": P.n, "box_m": [lx, ly], "particle_steps_per_s":
                                     P.n / (ms / 1e3), "ms_per_step": ms, "detection_ms": det_ms,
                                     "pairs_per_step": pairs / args.steps}
            del sim
    clk.window(t_clk, time.time())
    clk.__exit__()
    line = {"metric": "particle-steps/s of collision-only steps, plane sweep vs tree search",
            "unit": UNIT, "steps": args.steps, "warmup": args.warmup, "cases": rows,
            "data": "synthetic (seeded shearing-sheet generator)",
            "config": {"workload": f"no self-gravity, SEI, shear, eps=0.5; elongated box "
                                   f"{Lx:.0f} x {Ly:g} m with N={n:,}; square box "
                                   f"{L_SHEET:g} x {L_SHEET:g} m with N={N_SHEET:,}"}}
    line["clocks (whole run)"] = clk.summary()
    print(json.dumps(line), flush=True)
    return line


def _pairs_match(job):
    """Worker (spawned process): the oracle's Eq. 3 search on the GPU's
    end-of-step positions, compared with the GPU step's pair keys."""
    import oracle
    from paper_1110_4876_gb300 import inputs as I

    k, L, t, x, y, z, r, ids, keys = job
    p = oracle.Params(G=I.G_SI, omega=I.OMEGA, L=(L,) * 3, nghost=(1, 1, 0), boundary=2, integrator=1,
                      theta=0.5, eps=0.5, dt=I.DT_SHEET, gravity=1, collisions=1)
    ref = oracle.collide_tree(p, t, x, y, z, r, ids)
    return k, bool(np.array_equal(ref, keys)), len(keys), len(ref)


def run_precision(args):
    """The mid shearing sheet (N = 100,000, box 650 m, SEI, theta = 0.5,
    collisions eps = 0.5) for --precision-steps steps with the FP32 walk and
    with the FP64 walk: force errors against the oracle's FP64 tree (same
    theta) and its direct sum on 4096 seeded targets at the first, middle
    and last step; the collision pair set of every step against the
    oracle's search on the GPU's positions; the energy (Sect. 6.2) every 10
    steps.  One JSON line."""
    import multiprocessing

    nwork = max(1, min(32, (os.cpu_count() or 2) - 1))
    pool = multiprocessing.get_context("spawn").Pool(nwork)   # before any GPU call
    import torch

    import oracle
    from paper_1110_4876_gb300 import inputs as I
    from paper_1110_4876_gb300 import rb

    rb.load()
    stream = torch.cuda.Stream()
    L, n, nsteps = 650.0, 100_000, args.precision_steps
    P = I.sheet(L, n, 2)
    p = oracle.Params(G=I.G_SI, omega=I.OMEGA, L=(L,) * 3, nghost=(1, 1, 0), boundary=2, integrator=1,
                      theta=0.5, eps=0.5, dt=I.DT_SHEET, gravity=1, collisions=1)
    sel = np.random.default_rng(1).choice(n, 4096, replace=False)
    marks = sorted({0, nsteps // 2, nsteps})
    clk = Clocks(torch.cuda.current_device()).__enter__()
    t_start = time.time()
    forms = {}
    for walk in ("fp32", "fp64"):
        cfg = sheet_config(rb, walk)
        cfg["box"] = (L, L, L)
        sim = rb.Sim(stream=stream.cuda_stream, **cfg)
        sim.set_particles(P)
        rb.rb_autotune(sim.h)
        sim.set_particles(P)

        def errors(step):
            g = sim.particles()
            a = sim.gravity()
            t = oracle.time_at(p, 2 * step)
            a_tree = oracle.Tree(g["x"], g["y"], g["z"], g["m"], L).gravity(p, t, targets=sel)
            a_dir = oracle.direct_gravity(p, t, g["x"], g["y"], g["z"], g["m"], targets=sel)
            return {"vs_oracle_tree_same_theta": _errors(a[sel], a_tree),
                    "vs_direct_sum": _errors(a[sel], a_dir)}

        err = {0: errors(0)}
        E0, _ = sim.energy()
        energy = [(0, E0)]
        pending, results, step_ms = [], [], []
        for k in range(1, nsteps + 1):
            sim.step(1)
            step_ms.append(sim.stats()["ms_last_step"])
            g = sim.particles()
            keys = rb.pair_keys(*sim.pairs(detect=False))
            pending.append(pool.apply_async(_pairs_match, ((k, L, oracle.time_at(p, 2 * k), g["x"], g["y"],
                                                            g["z"], g["r"], g["id"], keys),)))
            while len(pending) > 4 * nwork:
                results.append(pending.pop(0).get())
            if k % 10 == 0:
                energy.append((k, sim.energy()[0]))
            if k in marks:
                err[k] = errors(k)
        results += [r.get() for r in pending]
        equal = sum(1 for r in results if r[1])
        forms[walk] = {
            "ms_per_step_device": statistics.mean(step_ms),
            "particle_steps_per_s_device": n / (statistics.mean(step_ms) / 1e3),
            "force_error": {f"step {k}": v for k, v in sorted(err.items())},
            "pair_sets": {"steps_checked": len(results), "steps_equal": equal,
                          "pairs_per_step": statistics.mean(r[2] for r in results),
                          "first_mismatch": next((r[0] for r in sorted(results) if not r[1]), None)},
            "energy": {"every": 10, "E0": E0,
                       "rel_drift": [(k, (E - E0) / abs(E0)) for k, E in energy]},
        }
        del sim
    clk.window(t_start, time.time())
    clk.__exit__()
    pool.close()
    pool.join()
    line = {"metric": "precision run: force error, pair-set equality and energy per walk form",
            "unit": "(see fields)", "steps": nsteps, "forms": forms, "clocks": clk.summary(),
            "data": "synthetic (seeded shearing-sheet generator)",
            "config": {"workload": f"shearing sheet N={n:,} box {L:g}x{L:g} m, 1 ghost ring, SEI, "
                                   f"theta=0.5 quadrupole, collisions eps=0.5, {nsteps} steps",
                       "targets": 4096, "oracle_workers": nwork,
                       "energy": "E = K + SEI tidal/vertical term + W (Sect. 6.2), W from the FP64 "
                                 "tree potential; collisions with eps = 0.5 dissipate energy"}}
    print(json.dumps(line), flush=True)
    return line


def _at_error(rows, target):
    """Throughput where a form's e_sum crosses `target`, interpolating
    log(e_sum) and throughput linearly in theta; None if it never does."""
    pts = sorted((r["theta"], r["force_error_vs_direct"]["e_sum"], r["particle_steps_per_s"]) for r in rows)
    for (t0, e0, v0), (t1, e1, v1) in zip(pts, pts[1:]):
        if e0 <= target <= e1 and e1 > e0:
            f = (math.log(target) - math.log(e0)) / (math.log(e1) - math.log(e0))
            return {"theta": t0 + f * (t1 - t0), "particle_steps_per_s": v0 + f * (v1 - v0)}
    if pts and abs(pts[0][1] - target) <= 1e-12 * target:
        return {"theta": pts[0][0], "particle_steps_per_s": pts[0][2]}
    return None


def run_learned_sweep(args):
    """The learned far-field correction against the plain FP32 walk on the
    1M sheet: the network trained once on ~10M residuals (two snapshots of
    the small and mid sheets), then e_sum / rms / max force error against
    the oracle's direct sum on 4096 targets and particle-steps/s of the full
    step for the plain walk at theta 0.5 ... 0.8 and the learned walk
    (fallback 0.5) at theta 0.6, 0.7, 0.8; and each form's throughput where
    its error equals the plain theta = 0.5 error.  One JSON line."""
    import torch

    import oracle
    from paper_1110_4876_gb300 import inputs as I
    from paper_1110_4876_gb300 import learned
    from paper_1110_4876_gb300 import rb

    rb.load()
    stream = torch.cuda.Stream()
    clk = Clocks(torch.cuda.current_device()).__enter__()
    t_clk = time.time()
    t = time.perf_counter()
    X, Y = learned.samples()
    t_samples = time.perf_counter() - t
    t = time.perf_counter()
    w, hist = rb.rb_mlp_train(X, Y, learned.init_weights(3), epochs=12, batch=2048, lr=1e-3, seed=1,
                              stream=stream.cuda_stream)
    t_train = time.perf_counter() - t
    batches = 12 * math.ceil(len(X) / 2048)
    P = I.sheet(L_SHEET, N_SHEET, SEED)
    sel = np.random.default_rng(1).choice(P.n, 4096, replace=False)
    p = oracle.Params(G=I.G_SI, omega=I.OMEGA, L=(L_SHEET,) * 3, nghost=(1, 1, 0), boundary=2,
                      integrator=1, theta=0.5, eps=0.5, dt=I.DT_SHEET, gravity=1, collisions=1)
    a_dir = oracle.direct_gravity(p, 0.0, P.x, P.y, P.z, P.m, targets=sel)
    forms = {"plain": [], "learned": []}
    for form, thetas in (("plain", (0.5, 0.55, 0.6, 0.65, 0.7, 0.75, 0.8)), ("learned", (0.6, 0.7, 0.8))):
        for theta in thetas:
            cfg = sheet_config(rb, "fp32" if form == "plain" else "learned")
            cfg["theta"] = theta
            sim = rb.Sim(stream=stream.cuda_stream, **cfg)
            if form == "learned":
                rb.rb_load_mlp(sim.h, w, 0.5)
            sim.set_particles(P)
            a = sim.gravity()
            err = _errors(a[sel], a_dir)
            corr = sim.stats()["corrections"]
            sim.set_particles(P)
            ms, wms, shape = _timed(sim, stream, args.steps, args.warmup)
            forms[form].append({"theta": theta, "particle_steps_per_s": N_SHEET / (ms / 1e3),
                                "ms_per_step": ms, "walk_ms": wms, "force_error_vs_direct": err,
                                "launch_shape": shape,
                                "corrected_cells_per_particle": corr / N_SHEET if form == "learned" else 0})
            del sim
    target = forms["plain"][0]["force_error_vs_direct"]["e_sum"]
    clk.window(t_clk, time.time())
    clk.__exit__()
    line = {"metric": "learned far-field correction vs plain FP32 walk: force error and particle-steps/s",
            "unit": UNIT, "steps": args.steps, "warmup": args.warmup, "forms": forms,
            "equal_error": {"target_e_sum (plain theta=0.5)": target,
                            "plain": _at_error(forms["plain"], target),
                            "learned": _at_error(forms["learned"], target)},
            "training": {"rows": len(X), "epochs": 12, "batch": 2048, "batches": batches,
                         "sampling_s": t_samples, "training_s": t_train,
                         "ms_per_batch": 1e3 * t_train / batches,
                         "loss_per_epoch": [float(v) for v in hist],
                         "recipe": "residuals of cells accepted at theta 0.8 with w/R > 0.5, two "
                                   "snapshots (0 and 50 steps) of the 100 m / 2400 and 650 m / "
                                   "100,000 sheets, kept fractions 1 and 0.42"},
            "clocks (whole run)": clk.summary(),
            "data": "synthetic (seeded shearing-sheet generator)",
            "config": {"workload": workload_name("fp32").replace("theta=0.5 quadrupole, fp32 walk",
                                                                 "theta swept, quadrupole"),
                       "targets": 4096}}
    print(json.dumps(line), flush=True)
    return line


def run_oracle_step(args):
    """One whole oracle step of the 1M sheet on this host (OMP_NUM_THREADS
    sets the threads), timed; one JSON line."""
    from paper_1110_4876_gb300 import inputs as I

    P = I.sheet(L_SHEET, N_SHEET, SEED)
    secs, npairs, cores = oracle_full_step(P)
    line = {"metric": "oracle step time (whole DKD step, FP64, host cores)", "unit": "s",
            "value": secs, "particle_steps_per_s": P.n / secs, "threads": cores, "pairs": npairs,
            "config": {"workload": workload_name("fp64 oracle"), "particles": P.n}}
    print(json.dumps(line), flush=True)
    return line


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return None
    from paper_1110_4876_gb300 import inputs as I

    P = I.sheet(L_SHEET, N_SHEET, SEED)
    times = []
    detail = cores = None
    for k in range(args.warmup + args.steps):
        per, detail, cores, _, _ = oracle_sample(P, args.cpu_samples // 4, seed=k)
        if k >= args.warmup:
            times.append(per)
    per = statistics.mean(times)
    value = 1.0 / per
    line = {"metric": METRIC, "value": value, "unit": UNIT, "impl": "reference", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": per * N_SHEET * 1e3,
            "ms_per_step_basis": "extrapolated: each timed step is a bounded sample (drifts and "
                                 "tree builds on all particles, walk and search from random "
                                 "targets) whose per-particle cost is scaled to N; a whole oracle "
                                 "step is timed by the default run's cpu_baseline",
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded shearing-sheet generator)",
            "config": {"workload": workload_name("fp64 oracle"), "particles": N_SHEET},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": detail},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return line


def main():
    global N_SHEET, L_SHEET
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawTextHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--walk", choices=["fp32", "fp64", "learned"], default="fp32",
                    help="fp32 / fp64 walk at theta 0.5, or the learned correction at theta 0.8")
    ap.add_argument("--cpu-samples", type=int, default=16384)
    ap.add_argument("--shape", type=lambda v: [int(x) for x in v.split(",")], default=None,
                    help="walk block, search block, walk group, tile order (default: autotuned); "
                         "fixes the kernels a profiler captures")
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--particles", type=int, default=N_SHEET,
                    help="sheet size (default 1M; smaller sizes are for profiling only)")
    ap.add_argument("--box", type=float, default=L_SHEET, help="sheet side in m (default 2050)")
    ap.add_argument("--ensemble", action="store_true",
                    help="measure the 256-box ensemble (batched vs looped) instead")
    ap.add_argument("--compare", action="store_true",
                    help="each walk form on the 1M sheet with its force error vs direct sum")
    ap.add_argument("--extensions", action="store_true",
                    help="the 1M sheet with the power-law restitution and with test particles")
    ap.add_argument("--plummer", action="store_true",
                    help="FP32 and FP64 walks on the 2^20 Plummer sphere at theta 0.3/0.5/0.7")
    ap.add_argument("--sweep", action="store_true",
                    help="plane sweep vs tree search on collision-only elongated and square sheets")
    ap.add_argument("--cases", default="elongated,square", help="--sweep cases to run")
    ap.add_argument("--precision", action="store_true",
                    help="100k sheet, FP32 and FP64 walks: force errors, per-step pair sets, energy")
    ap.add_argument("--precision-steps", type=int, default=1000)
    ap.add_argument("--oracle-step", action="store_true",
                    help="time one whole oracle step of the 1M sheet on the host (OMP_NUM_THREADS)")
    ap.add_argument("--learned-sweep", action="store_true",
                    help="learned vs plain FP32 walk over theta on the 1M sheet, at equal error")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    N_SHEET, L_SHEET = args.particles, args.box
    if args.impl == "reference":
        run_reference(args)
    elif args.ensemble:
        run_ensemble(args)
    elif args.compare:
        run_compare(args)
    elif args.extensions:
        run_extensions(args)
    elif args.plummer:
        run_plummer(args)
    elif args.sweep:
        run_sweep(args)
    elif args.precision:
        run_precision(args)
    elif args.learned_sweep:
        run_learned_sweep(args)
    elif args.oracle_step:
        run_oracle_step(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
