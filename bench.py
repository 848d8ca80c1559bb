#!/usr/bin/env python3
"""Benchmark: Barnes-Hut particle-steps/s on one GB300 (or N replicas).

Default workload (one "step" = one kick-drift-kick leapfrog step, i.e. one
pass of the whole hot path: bounding box, Morton keys, radix sort, octree
topology, centre-of-mass pass, walk, kicks): a uniform cube of N = 1,048,576
particles U[-1,1]^3, zero velocities, masses 1/N, G = 1, eps = 0.005,
theta = 0.5, dt = 5e-4, FP32 walk with FP64 root reductions, seed 2.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line.  Device time comes from CUDA events the library records
on its own stream around each phase of each step (integrate, build, walk); L2
is flushed between timed steps (outside the timed events).  For N > 1 (launched
by torch.distributed.run) every rank runs an independent replica; the value is
the particle-steps of all ranks over the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Barnes-Hut particle-steps/s batched vs plain at force err≤1e-4; p50/p99 latency"
UNIT = "particle-steps/s"
WORKLOAD = ("uniform cube N=1,048,576 U[-1,1]^3, v=0, m=1/N, G=1, eps=0.005, theta=0.5, "
            "dt=5e-4 KDK leapfrog, FP32 walk (Kahan) + FP64 root reductions, seed 2")
N_PART = 1 << 20
THETA, EPS, DT, SEED = 0.5, 0.005, 5e-4, 2
KIND = "uniform"
WORKLOADS = {
    # the headline workload (default)
    "uniform1m": dict(N_PART=1 << 20, THETA=0.5, EPS=0.005, DT=5e-4, SEED=2, KIND="uniform",
                      WORKLOAD=WORKLOAD),
    # the large single Plummer sphere, selectable as the main leg (for profiling)
    "large": dict(N_PART=1 << 24, THETA=0.6, EPS=0.002, DT=2.5e-4, SEED=3, KIND="plummer",
                  WORKLOAD="Plummer N=16,777,216, m=1/N, G=1, eps=0.002, theta=0.6, "
                           "dt=2.5e-4 KDK leapfrog, FP32 walk (Kahan) + FP64 root reductions, seed 3"),
}


def make_inputs():
    import synth
    if KIND == "plummer":
        return synth.plummer(N_PART, SEED)
    return synth.uniform_cube(N_PART, SEED)
FLOPS_PER_INTERACTION = 20


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    """nvidia-smi samples (every 25 ms: the timed region of the default run is
    well under a second) of SM clock and throttle reasons."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "25"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2] if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def combine_ranks(local_ms: float, units_per_rank: int, steps: int, device=None):
    """(slowest rank's time in ms, whole-job units/s): every rank ran `steps`
    steps of `units_per_rank` units; max over ranks, no data-path collective
    beyond this one scalar."""
    import torch
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    t_max = float(local_ms)
    if ws > 1:
        import torch.distributed as dist
        tt = torch.tensor([t_max], dtype=torch.float64, device=device)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t_max = float(tt.item())
    return t_max, ws * units_per_rank * steps / (t_max * 1e-3)


def shard_of(B, sizes, world: int, rank: int):
    """Indices of the systems `rank` runs when independent systems of the
    given sizes are dealt to `world` ranks (bh_partition_systems)."""
    r = B.bh_partition_systems(sizes, world)
    return [k for k in range(len(sizes)) if int(r[k]) == rank]


def over_ranks(x: float, op: str = "max", device=None) -> float:
    """A host scalar reduced over the ranks (max or sum); x itself on one rank."""
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws == 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def code_digest(texts) -> str:
    """SHA-256 of C/CUDA sources with comments and whitespace removed, so that
    it changes with the code and not with its comments."""
    import hashlib
    import re
    h = hashlib.sha256()
    for t in texts:
        t = re.sub(r"/\*.*?\*/", "", t, flags=re.S)
        t = re.sub(r"//[^\n]*", "", t)
        h.update(re.sub(r"\s+", "", t).encode())
    return h.hexdigest()


def walk_sources_sha() -> str:
    """Code digest of the walk's sources (walk.cu and the shared header)."""
    texts = []
    for f in ("walk.cu", "bh_internal.cuh"):
        with open(os.path.join(ROOT, "paper_1109_5190_gb300", "csrc", f)) as fh:
            texts.append(fh.read())
    return code_digest(texts)


def walk_profile_field(name: str):
    """An integer field (DRAM bytes, L1 sectors per walk launch) of the
    committed ncu capture summary of the walk, or None once the walk's sources
    differ from the ones that capture measured."""
    path = os.path.join(ROOT, "profiles", "walk_uniform1M_ncu.md")
    try:
        text = open(path).read()
    except OSError:
        return None
    fields = dict(line.split(":", 1) for line in text.splitlines()
                  if line.startswith(("walk_source_sha256:", name + ":")))
    if fields.get("walk_source_sha256", "").strip() != walk_sources_sha():
        return None
    try:
        return int(fields[name].strip())
    except (KeyError, ValueError):
        return None


def walk_traffic():
    """DRAM bytes per walk launch (committed ncu capture), or None."""
    return walk_profile_field("dram_bytes_per_launch")


# ---------------------------------------------------------------- reference

def cpu_sample(pm, sample: int, seed: int = 7):
    """Oracle (FP64 CPU Barnes-Hut) on a bounded sample of one step: the full
    tree build plus the walk of `sample` particles, extrapolated to all N.
    Returns (particle-steps/s, seconds spent, threads)."""
    import numpy as np
    import oracle
    n = len(pm)
    threads = os.cpu_count() or 1
    t0 = time.perf_counter()
    T = oracle.Tree(pm)
    t1 = time.perf_counter()
    idx = np.random.default_rng(seed).choice(n, min(sample, n), replace=False)
    T.accel(THETA, EPS, targets=idx, nthreads=threads)
    t2 = time.perf_counter()
    t_step = (t1 - t0) + (t2 - t1) * n / len(idx)
    return n / t_step, t2 - t0, threads


def cpu_one_core(pm, sample: int = 4096, seed: int = 8):
    """The same oracle step with the walk on one thread (a smaller sample):
    (particle-steps/s, seconds spent)."""
    import numpy as np
    import oracle
    n = len(pm)
    t0 = time.perf_counter()
    T = oracle.Tree(pm)
    t1 = time.perf_counter()
    idx = np.random.default_rng(seed).choice(n, min(sample, n), replace=False)
    T.accel(THETA, EPS, targets=idx, nthreads=1)
    t2 = time.perf_counter()
    return n / ((t1 - t0) + (t2 - t1) * n / len(idx)), t2 - t0


def cpu_model() -> str:
    """The host CPU's model name (lscpu), else the machine type."""
    import platform
    import subprocess
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    return platform.machine()


def oracle_errors(pos_mass, acc, theta, eps, sample=4096, seed=11, G=1.0):
    """Force error of one result against the FP64 oracle, outside every timed
    region: the oracle's tree of all of pos_mass, walked for a seeded sample of
    particles.  Returns dict(err_p99, err_max, sample): the 99th percentile of
    |a - a_ref| / |a_ref| and the maximum of |a - a_ref| / max(|a_ref|,
    1e-3 rms|a_ref|) over the sample (rms over the sample), the measures the
    parity tests gate at 1e-5 and 1e-3."""
    import numpy as np
    import oracle
    n = len(pos_mass)
    idx = np.sort(np.random.default_rng(seed).choice(n, min(sample, n), replace=False))
    ref, _, _ = oracle.Tree(pos_mass).accel(theta, eps, G, targets=idx,
                                             nthreads=os.cpu_count() or 1)
    a = np.asarray(acc, dtype=np.float64)[idx, :3]
    d = np.linalg.norm(a - ref, axis=1)
    r = np.linalg.norm(ref, axis=1)
    rms = float(np.sqrt(np.mean(r * r)))
    rel = np.where(d > 0, d / np.where(r > 0, r, 1.0), 0.0)
    relmax = np.where(d > 0, d / np.maximum(r, 1e-3 * rms), 0.0)
    return {"err_p99": float(np.percentile(rel, 99)), "err_max": float(relmax.max()),
            "err_sample": f"{len(idx)} of {n} particles (seed {seed}), FP64 oracle tree of all {n}"}


def system_errors(B, h, n, theta, eps, sample=4096, seed=11):
    """oracle_errors of a single system's current state (bh_get_state)."""
    import numpy as np
    x = np.zeros((n, 4), np.float32)
    a = np.zeros((n, 4), np.float32)
    B.bh_get_state(h, x, None, a)
    return oracle_errors(x, a, theta, eps, sample, seed)


def run_reference(args):
    """The oracle as it stands, timed on the host cores.  Each step builds the
    FP64 tree of all N particles and walks a sample of them; the sample is the
    whole system when the run fits args.ref_budget_s seconds, else the largest
    share that does, and the value is then extrapolated to all N (the line says
    which)."""
    import numpy as np
    import oracle
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    pm, _ = make_inputs()
    n = len(pm)
    threads = os.cpu_count() or 1
    # size the per-step sample from one probe step (tree + 4096-particle walk)
    t0 = time.perf_counter()
    T = oracle.Tree(pm)
    t1 = time.perf_counter()
    probe = np.random.default_rng(99).choice(n, min(4096, n), replace=False)
    T.accel(THETA, EPS, targets=probe, nthreads=threads)
    t2 = time.perf_counter()
    del T
    per_particle = (t2 - t1) / len(probe)
    per_step_budget = args.ref_budget_s / max(args.steps, 1)
    sample = int(min(n, max(4096, (per_step_budget - (t1 - t0)) / max(per_particle, 1e-12))))
    vals, spent, walk_s, tree_s = [], 0.0, 0.0, 0.0
    for k in range(args.warmup + args.steps):
        timed = k >= args.warmup
        s_k = sample if timed else min(4096, n)
        idx = np.arange(n) if s_k >= n else \
            np.random.default_rng(100 + k).choice(n, s_k, replace=False)
        a0 = time.perf_counter()
        T = oracle.Tree(pm)
        a1 = time.perf_counter()
        T.accel(THETA, EPS, targets=idx, nthreads=threads)
        a2 = time.perf_counter()
        del T
        if timed:
            spent += a2 - a0
            tree_s += a1 - a0
            walk_s += a2 - a1
            vals.append(n / ((a1 - a0) + (a2 - a1) * n / len(idx)))
    value = len(vals) / sum(1.0 / v for v in vals)  # total particle-steps / total time
    full = sample >= n
    how = ("each timed step: full FP64 tree build of all {n} particles (1 thread) + walk of "
           "all {n} particles ({t} threads): measured, not extrapolated" if full else
           "each timed step: full FP64 tree build of all {n} particles (1 thread) + walk of "
           "{s} random particles ({t} threads), walk time extrapolated to all {n}").format(
               n=n, s=sample, t=threads)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * n / value,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": n, "extrapolated": not full,
                   "walk_sample_per_step": sample},
        "measured_s": {"timed_steps_total": spent, "tree": tree_s, "walk": walk_s},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": how, "cpu_model": cpu_model()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------- GPU

def run_gpu(args):
    import numpy as np
    import torch

    import synth
    from paper_1109_5190_gb300 import binding as B

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()

    pm, vel = make_inputs()
    d_pm = torch.from_numpy(pm).to(dev)
    d_vel = torch.from_numpy(vel).to(dev)
    flags = B.BH_NO_KAHAN if args.no_kahan else 0
    h = B.bh_create(B.params(1.0, EPS, THETA, flags), d_pm, d_vel, stream)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # > 129 MB L2

    if args.ppl:
        B.bh_set_tuning(h, args.ppl, args.warps, args.bps, args.group, args.static_share)
        tuning = B.bh_get_tuning(h)
    else:
        tuning = B.bh_autotune(h)
    B.bh_compute_accel(h)
    graph = not args.no_graph
    B.bh_profile_begin(h)  # the captured step then carries its phase events
    for _ in range(args.warmup):
        B.bh_step(h, 1, DT, graph)
    B.bh_profile_end(h)
    ws0 = B.bh_walk_stats(h)
    inter0 = ws0["interactions"]

    sampler = ClockSampler(local)
    sampler.start()
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    B.bh_profile_begin(h)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        flush.fill_(1)
        torch.cuda.synchronize()
        B.bh_step(h, 1, DT, graph)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    phase_ms, nsteps, launches = B.bh_profile_end(h)
    clocks = sampler.stop()
    ws1 = B.bh_walk_stats(h)
    inter1 = ws1["interactions"]
    dev_ms = float(phase_ms.sum())
    if nsteps != args.steps or dev_ms <= 0:
        raise RuntimeError(f"phase events recorded {nsteps} steps / {dev_ms} ms for {args.steps} steps")

    t_max, value = combine_ranks(dev_ms, N_PART, args.steps, dev)

    # ---- roofline of the dominant kernel (the walk): FP32 ALU bound
    walk_ms = phase_ms[2] / nsteps
    inter = 0.5 * (inter0 + inter1)
    achieved = inter * FLOPS_PER_INTERACTION / (walk_ms * 1e-3) / 1e12
    fma_peak = B.bh_micro_fma_peak(stream) / 1e3
    l1_peak = B.bh_micro_l1_gather(stream)  # G sectors/s
    l1_sectors = walk_profile_field("l1_sectors_per_launch")
    peaks, peak_src = measured_peaks()
    build_ms = phase_ms[1] / nsteps
    # algorithmic bytes of the build: 144 B per particle + 48 B per node
    n_nodes = B.bh_node_count(h)
    build_bytes = 144 * N_PART + 48 * n_nodes
    build_gbs = build_bytes / (build_ms * 1e-3) / 1e9
    # error of the state the timed steps reached, against the FP64 oracle
    errs = system_errors(B, h, N_PART, THETA, EPS) if rank == 0 else {}

    # ---- end to end through the C ABI with host buffers
    e2e = None
    if not args.no_e2e:
        hpm = torch.empty((N_PART, 4), dtype=torch.float32, pin_memory=True).numpy()
        hvel = torch.empty_like(torch.from_numpy(hpm)).pin_memory().numpy()
        hacc = torch.empty_like(torch.from_numpy(hpm)).pin_memory().numpy()
        B.bh_get_state(h, hpm, hvel, hacc)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            B.bh_set_state(h, hpm, hvel, hacc)
            B.bh_step(h, 1, DT, graph)  # the same step graph as the device-timed loop
            B.bh_get_state(h, hpm, hvel, hacc)
        e2e_s = time.perf_counter() - t0
        e2e = {"value": N_PART * args.steps * ws / e2e_s, "unit": UNIT,
               "h2d_bytes_per_step": 3 * N_PART * 16, "d2h_bytes_per_step": 3 * N_PART * 16}

    B.bh_destroy(h)
    extra = {}
    if rank == 0 and not args.no_theta07 and args.workload == "uniform1m":
        extra["theta_0.7"] = bench_other_theta(args, B, torch, 0.7)
    # sharded by system over every rank (one rank: the whole workload)
    if not args.no_batched:
        extra["batched"] = bench_batched(args, B, torch, dev)
    if not args.no_served:
        extra["served"] = bench_served(args, B, torch, dev)
    if rank == 0 and not args.no_large:
        extra["large"] = bench_large(args, B, torch, fma_peak, peaks["hbm_gbs"])

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": N_PART, "theta": THETA, "eps": EPS, "dt": DT,
                   "parallelism": f"replicas{ws}" if ws > 1 else "single",
                   "l2": "flushed between timed steps (256 MiB write, outside the timed events)",
                   "walk_shape": {"ppl": tuning[0], "warps_per_block": tuning[1],
                                  "blocks_per_sm": tuning[2], "group": tuning[3],
                                  "static_share": tuning[4]}},
        "phase_ms_per_step": {"integrate": phase_ms[0] / nsteps, "build": build_ms, "walk": walk_ms},
        "wall_ms_per_step": 1e3 * wall / args.steps,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": fma_peak, "unit": "TFLOP/s",
                     "frac": achieved / fma_peak, "traffic": walk_traffic(),
                     "kernel": "k_walk", "peak_source": "project FP32 FMA micro-benchmark",
                     "interactions_per_launch": inter, "flops_per_interaction": FLOPS_PER_INTERACTION,
                     "warp_iterations_per_launch": ws1["warp_iterations"],
                     "lane_efficiency": ws1["interactions"] / (32.0 * ws1["warp_iterations"]),
                     "slot_visits_per_launch": ws1["slot_visits"]},
        # the walk against the limit it meets first: L1 throughput for
        # scattered 32-byte node loads (project micro-benchmark), sectors per
        # launch from the committed ncu capture of the same walk
        "l1_roofline": {"bound": "l1", "unit": "G sectors/s", "peak": l1_peak,
                        "achieved": (l1_sectors / (walk_ms * 1e-3) / 1e9) if l1_sectors else None,
                        "frac": (l1_sectors / (walk_ms * 1e-3) / 1e9 / l1_peak) if l1_sectors else None,
                        "sectors_per_launch": l1_sectors, "kernel": "k_walk",
                        "peak_source": "project micro-benchmark: each lane loads its own random "
                                       "32-byte record from an L1-resident table, 48 warps/SM"},
        "build_roofline": {"bound": "hbm", "achieved": build_gbs, "peak": peaks["hbm_gbs"],
                           "unit": "GB/s", "frac": build_gbs / peaks["hbm_gbs"],
                           "algorithmic_bytes": build_bytes, "nodes": n_nodes,
                           "peak_source": f"MEASURED_PEAKS.json hbm_gbs ({peak_src})"},
        "e2e": e2e,
        "clocks": clocks,
        "gpu_launches": launches,
    }
    line.update(errs)
    line.update(extra)
    if rank == 0 and ws == 1 and not args.no_cpu:
        v, spent, threads = cpu_sample(pm, args.cpu_sample)
        v1, spent1 = cpu_one_core(pm)
        walked = (f"walk of all {N_PART} particles ({threads} threads), timed in full"
                  if args.cpu_sample >= N_PART else
                  f"walk of {args.cpu_sample} random particles ({threads} threads), "
                  f"extrapolated to N")
        line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle",
                                "sample": f"one step: full FP64 tree build of {N_PART} particles "
                                          f"(1 thread) + {walked}; {spent:.1f} s",
                                "one_core_value": v1,
                                "one_core_sample": f"the same step with a 4096-particle walk on "
                                                   f"1 thread, extrapolated to N; {spent1:.1f} s",
                                "cpu_model": cpu_model()}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def bench_batched(args, B, torch, device=None):
    """Forest of many uneven systems (N log-uniform in [256, 65536], half
    Plummer, half uniform cold collapse, eps 0.01, theta 0.5, dt 1e-3): all
    steps of one call in one CUDA graph, one persistent walk per step across
    all trees; against the plain single-system path solving the same systems
    one after another.  With several ranks the systems are dealt to them by
    bh_partition_systems; each rank runs its share as its own forest, and the
    value is all ranks' particle-steps over the slowest rank's time."""
    import numpy as np

    import synth
    ws, rank, _ = dist_env()
    all_systems = synth.forest_systems(args.forest_systems, 256, 65536, seed=4, theta=0.5, eps=0.01)
    mine = shard_of(B, [s.n for s in all_systems], ws, rank)
    systems = [all_systems[k] for k in mine]
    n_tot = sum(s.n for s in systems)
    descs = [dict(pos_mass=s.pos_mass, vel=s.vel, eps=s.eps, theta=s.theta, dt=1e-3) for s in systems]
    f = B.bh_forest_create(descs)
    try:
        B.bh_forest_compute_accel(f)
        shape = B.bh_forest_autotune(f)
        B.bh_forest_step(f, args.forest_steps, 1e-3, True)  # capture + warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        B.bh_forest_step(f, args.forest_steps, 1e-3, True)
        torch.cuda.synchronize()
        t_forest = time.perf_counter() - t0
        _, nodes = B.bh_forest_info(f)
        # the same graph recaptured with phase events, run once more
        B.bh_forest_profile_begin(f)
        B.bh_forest_step(f, args.forest_steps, 1e-3, True)
        phase_ms, nst, _ = B.bh_forest_profile_end(f)
        # error against the oracle (rank 0): every particle of 8 seeded systems
        pick = sorted(np.random.default_rng(12).choice(len(systems), min(8, len(systems)),
                                                       replace=False).tolist())
        e99, emax = [], []
        for k in (pick if rank == 0 else []):
            sy = systems[k]
            x = np.zeros((sy.n, 4), np.float32)
            a = np.zeros((sy.n, 4), np.float32)
            B.bh_forest_get_state(f, k, x, None, a)
            e = oracle_errors(x, a, sy.theta, sy.eps, sample=sy.n)
            e99.append(e["err_p99"])
            emax.append(e["err_max"])
    finally:
        B.bh_forest_destroy(f)
    t_forest = over_ranks(t_forest, "max", device)
    n_all = int(over_ranks(n_tot, "sum", device))
    batched = n_all * args.forest_steps / t_forest
    # the plain path, one system after another (host wall time of bh_step
    # only), with its kernels launched directly and with its steps replayed
    # from a captured graph (captured by an untimed first call)
    t_plain, t_graph, ps_plain = 0.0, 0.0, 0
    for sy in systems:
        h = B.bh_create(B.params(1.0, sy.eps, sy.theta), sy.pos_mass, sy.vel)
        try:
            B.bh_compute_accel(h)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            B.bh_step(h, args.plain_steps, 1e-3)
            t_plain += time.perf_counter() - t0
            B.bh_step(h, args.plain_steps, 1e-3, True)  # capture + warm-up
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            B.bh_step(h, args.plain_steps, 1e-3, True)
            t_graph += time.perf_counter() - t0
            ps_plain += sy.n * args.plain_steps
        finally:
            B.bh_destroy(h)
    ps_plain = over_ranks(ps_plain, "sum", device)
    plain = ps_plain / over_ranks(t_plain, "max", device)
    plain_graph = ps_plain / over_ranks(t_graph, "max", device)
    return {"workload": f"{len(all_systems)} systems, N log-uniform [256, 65536] (sum {n_all}), "
                        "half Plummer / half uniform cold collapse, eps 0.01, theta 0.5, dt 1e-3, seed 4",
            "value": batched, "unit": UNIT, "steps_in_one_graph": args.forest_steps,
            "ranks": ws, "scaling": "strong",
            "sharding": "systems dealt to ranks by bh_partition_systems (n log2 n, longest "
                        "first); each rank runs its share as one forest; no data-path collective"
                        if ws > 1 else "single rank",
            "ms_per_step": 1e3 * t_forest / args.forest_steps, "nodes": nodes,
            "phase_ms_per_step": {k: float(v) / max(nst, 1) for k, v in
                                  zip(("integrate", "build", "walk"), phase_ms)},
            "walk_shape": list(shape),
            "err_p99": max(e99) if e99 else None, "err_max": max(emax) if emax else None,
            "err_sample": f"every particle of systems {[mine[k] for k in pick]} after "
                          f"{3 * args.forest_steps} graph steps, worst system reported, FP64 oracle"
                          + (" (rank 0's share)" if ws > 1 else ""),
            "plain_sequential": {"value": plain, "unit": UNIT,
                                 "steps_per_system": args.plain_steps,
                                 "how": "bh_step on each system in turn, kernels launched directly"},
            "plain_sequential_graph": {"value": plain_graph, "unit": UNIT,
                                       "steps_per_system": args.plain_steps,
                                       "how": "bh_step on each system in turn, its steps replayed "
                                              "from a CUDA graph captured by an untimed first call"},
            "speedup_vs_plain": batched / plain_graph,
            "speedup_vs_plain_direct_launches": batched / plain}


def bench_other_theta(args, B, torch, theta):
    """The headline workload (uniform cube of 2^20 particles, eps 0.005, dt
    5e-4) at another opening angle: the same KDK steps from a captured graph,
    autotuned, device time from the library's phase events."""
    pm, vel = make_inputs()
    d_pm = torch.from_numpy(pm).cuda()
    d_vel = torch.from_numpy(vel).cuda()
    h = B.bh_create(B.params(1.0, EPS, theta), d_pm, d_vel, torch.cuda.current_stream())
    del d_pm, d_vel
    try:
        shape = B.bh_autotune(h)
        B.bh_compute_accel(h)
        B.bh_profile_begin(h)
        B.bh_step(h, 1, DT, True)  # capture + warm-up
        B.bh_profile_end(h)
        torch.cuda.synchronize()
        B.bh_profile_begin(h)
        for _ in range(args.steps):
            B.bh_step(h, 1, DT, True)
        phase_ms, nst, _ = B.bh_profile_end(h)
        stats = B.bh_walk_stats(h)
        errs = system_errors(B, h, N_PART, theta, EPS)
    finally:
        B.bh_destroy(h)
    step_ms = float(phase_ms.sum()) / nst
    return {**errs, "workload": WORKLOAD.replace(f"theta={THETA}", f"theta={theta}"),
            "value": N_PART / (step_ms * 1e-3),
            "unit": UNIT, "ms_per_step": step_ms,
            "phase_ms_per_step": {k: float(v) / nst for k, v in
                                  zip(("integrate", "build", "walk"), phase_ms)},
            "walk_shape": list(shape),
            "interactions_per_particle": stats["interactions"] / N_PART}


def bench_large(args, B, torch, fma_peak_tflops, hbm_gbs):
    """Large single Plummer sphere: N = 16,777,216, masses 1/N, eps 0.002,
    theta 0.6, 10 KDK steps dt 2.5e-4 (FP32 positions/velocities/forces, Kahan
    force sums).  Build GB/s and walk interactions/s against their rooflines."""
    import synth
    n, theta, eps, dt, steps = 1 << 24, 0.6, 0.002, 2.5e-4, 10
    pm, vel = synth.plummer(n, 3)
    d_pm = torch.from_numpy(pm).cuda()
    d_vel = torch.from_numpy(vel).cuda()
    del pm, vel
    h = B.bh_create(B.params(1.0, eps, theta), d_pm, d_vel, torch.cuda.current_stream())
    del d_pm, d_vel
    try:
        shape = B.bh_autotune(h)
        B.bh_compute_accel(h)
        B.bh_profile_begin(h)
        B.bh_step(h, 1, dt, True)  # capture + warm-up
        B.bh_profile_end(h)
        stats = B.bh_walk_stats(h)
        nodes = B.bh_node_count(h)
        torch.cuda.synchronize()
        B.bh_profile_begin(h)
        for _ in range(steps):
            B.bh_step(h, 1, dt, True)
        phase_ms, nst, _ = B.bh_profile_end(h)
        errs = system_errors(B, h, n, theta, eps) if args.large_errors else {}
    finally:
        B.bh_destroy(h)
    walk_ms = phase_ms[2] / nst
    build_ms = phase_ms[1] / nst
    step_ms = float(phase_ms.sum()) / nst
    inter_s = stats["interactions"] / (walk_ms * 1e-3)
    build_gbs = (144 * n + 48 * nodes) / (build_ms * 1e-3) / 1e9
    return {**errs,
            "workload": "Plummer N=16,777,216, m=1/N, eps=0.002, theta=0.6, 10 KDK steps dt=2.5e-4, seed 3",
            "value": n / (step_ms * 1e-3), "unit": UNIT, "ms_per_step": step_ms,
            "phase_ms_per_step": {"integrate": phase_ms[0] / nst, "build": build_ms, "walk": walk_ms},
            "walk_shape": list(shape), "nodes": nodes,
            "walk_interactions_per_s": inter_s,
            "interactions_per_particle": stats["interactions"] / n,
            "walk_roofline": {"bound": "alu", "achieved": inter_s * FLOPS_PER_INTERACTION / 1e12,
                              "peak": fma_peak_tflops, "unit": "TFLOP/s",
                              "frac": inter_s * FLOPS_PER_INTERACTION / 1e12 / fma_peak_tflops},
            "build_roofline": {"bound": "hbm", "achieved": build_gbs, "peak": hbm_gbs, "unit": "GB/s",
                               "frac": build_gbs / hbm_gbs}}


def serve_pools():
    import synth
    return {"plummer": synth.plummer(1 << 21, 51), "uniform": synth.uniform_cube(1 << 21, 52)}


def serve_stream(B, rate_hz, seconds, seed, pools, full_seconds=60.0, check=8, device=None,
                 budget_gb=160.0):
    """Poisson request stream through bh_submit / bh_wait with continuous
    batching under an HBM budget (160 GB by default); each request a Plummer or uniform system
    of N log-uniform in [1024, 2097152], theta U[0.5, 0.8], 10-200 KDK steps of
    dt 1e-3, eps 0.01.  A request's particles are a window of consecutive
    particles (at a seeded offset, wrapping around) of a pre-drawn 2^21-particle
    Plummer sphere or uniform cube of independent draws, masses 1/N; payloads
    are made up front, or as the requests arrive when a long window would hold
    too much host memory.  With several ranks the requests are dealt to them by
    bh_partition_systems (on N x steps) and each rank serves its share with its
    own server; latencies are gathered on the host.  Results of `check` seeded
    requests with N <= 2^18 are checked against the FP64 oracle (rank 0)."""
    import numpy as np
    import synth
    ws, rank, _ = dist_env()
    all_reqs = synth.request_stream(rate_hz=rate_hz, duration_s=seconds, seed=seed)
    mine = shard_of(B, [r.n * max(r.steps, 1) for r in all_reqs], ws, rank)
    reqs = [all_reqs[k] for k in mine]
    small = [k for k, r in enumerate(reqs) if r.n <= 1 << 18] if rank == 0 else []
    checked = set(np.random.default_rng(seed + 1000).choice(
        small, min(check, len(small)), replace=False).tolist()) if small else set()

    def payload(r):
        rng = np.random.default_rng(r.seed)
        pm_pool, v_pool = pools[r.kind]
        idx = np.arange(r.n) + int(rng.integers(0, len(pm_pool)))
        pm = np.ascontiguousarray(np.take(pm_pool, idx, axis=0, mode="wrap"))
        pm[:, 3] = np.float32(1.0 / r.n)
        return pm, np.ascontiguousarray(np.take(v_pool, idx, axis=0, mode="wrap"))

    # made up front unless that would hold more than 8 GB of host memory
    ready = None
    if sum(r.n for r in reqs) * 32 <= 8 << 30:
        ready = [payload(r) for r in reqs]
    srv = B.bh_server_create(int(budget_gb * (1 << 30)), 256)
    tickets = [None] * len(reqs)
    try:
        t0 = time.perf_counter()

        failed = []

        def submit():
            try:
                for k, r in enumerate(reqs):
                    pm, v = ready[k] if ready is not None else payload(r)
                    delay = r.arrival_s - (time.perf_counter() - t0)
                    if delay > 0:
                        time.sleep(delay)
                    tickets[k] = B.bh_submit(srv, pm, v, 1.0, r.eps, r.theta, r.dt, r.steps)
            except Exception as e:  # the collector stops waiting for tickets
                failed.append(e)

        # results are collected in submission order while requests still
        # arrive, so finished requests do not pile up in host memory
        res = [None] * len(reqs)

        def collect():
            try:
                for k in range(len(reqs)):
                    while tickets[k] is None:
                        if failed:
                            return
                        time.sleep(1e-3)
                    res[k] = B.bh_wait(srv, tickets[k], reqs[k].n if k in checked else 0, 7200.0)
            except Exception as e:
                failed.append(e)

        th = threading.Thread(target=submit)
        tc = threading.Thread(target=collect)
        th.start()
        tc.start()
        th.join()
        tc.join()
        if failed:
            raise failed[0]
        if any(r is None for r in res):
            raise RuntimeError("a served request returned no result")
        stats = B.bh_server_stats_get(srv)
    finally:
        B.bh_server_destroy(srv)
    lat = [x["done_s"] - x["submit_s"] for x in res]
    ps = sum(r.n * r.steps for r in reqs)
    # each rank's span on its own server clock (all started within the same
    # second); the job's rate is all ranks' particle-steps over the longest span
    span = (max(x["done_s"] for x in res) - min(x["submit_s"] for x in res)) if res else 0.0
    if ws > 1:
        import torch.distributed as dist
        parts = [None] * ws
        dist.all_gather_object(parts, lat)
        lat = [v for p in parts for v in p]
        span = over_ranks(span, "max", device)
        ps = over_ranks(ps, "sum", device)
        stats = {k: over_ranks(stats[k], "sum", device) for k in
                 ("peak_resident_systems", "peak_resident_bytes", "ticks")} | \
                {"busy_s": over_ranks(stats["busy_s"], "max", device)}
    lat = np.array(lat)
    e99, emax = [], []
    for k in sorted(checked):
        e = oracle_errors(res[k]["pos_mass"], res[k]["acc"], reqs[k].theta, reqs[k].eps)
        e99.append(e["err_p99"])
        emax.append(e["err_max"])
    window = (f"{seconds} s of arrivals (the full stream)" if seconds >= full_seconds else
              f"truncated window: {seconds} s of arrivals, not the {full_seconds:g} s stream")
    return {"workload": f"{len(all_reqs)} requests, Poisson {rate_hz:.3g}/s, {window}, "
                        "N log-uniform [1024, 2097152], theta U[0.5,0.8], 10-200 steps dt 1e-3, "
                        f"Plummer/uniform 50/50, seed {seed}",
            "value": ps / span, "unit": UNIT, "p50_latency_s": float(np.percentile(lat, 50)),
            "p99_latency_s": float(np.percentile(lat, 99)),
            "offered_particle_steps_per_s": ps / max(seconds, 1e-9), "requests": len(all_reqs),
            "ranks": ws,
            "admitted_particle_steps_per_s": ps / span,
            "peak_resident_systems": stats["peak_resident_systems"],
            "peak_resident_bytes": stats["peak_resident_bytes"],
            "ticks": stats["ticks"], "busy_s": stats["busy_s"],
            "err_p99": max(e99) if e99 else None, "err_max": max(emax) if emax else None,
            "err_sample": f"{len(e99)} seeded requests with N <= 2^18, 4096 particles each, "
                          "FP64 oracle tree of the returned positions"}


def bench_served(args, B, torch, device=None):
    """The request stream of the served workload (200 requests/s), then the
    same mix at half the throughput the first run measured, where latency is
    service time rather than queueing."""
    pools = serve_pools()
    out = serve_stream(B, 200.0, args.serve_seconds, 5, pools, device=device,
                       budget_gb=args.serve_budget_gb)
    if args.serve_light_seconds > 0:
        per_request = out["offered_particle_steps_per_s"] / 200.0  # particle-steps per request
        rate = 0.5 * out["value"] / max(per_request, 1.0)
        light = serve_stream(B, rate, args.serve_light_seconds, 6, pools, device=device,
                             budget_gb=args.serve_budget_gb)
        light["load"] = "offered load = 0.5 x the throughput measured at 200 requests/s"
        out["half_load"] = light
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--cpu-sample", type=int, default=1 << 20)
    ap.add_argument("--ref-budget-s", type=float, default=120.0,
                    help="host seconds the reference arm's timed steps may take; the per-step "
                         "walk sample is sized to fit (the whole system when it does)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--ppl", type=int, default=0, help="fix the walk shape (skip the autotuner)")
    ap.add_argument("--warps", type=int, default=8)
    ap.add_argument("--bps", type=int, default=0, help="walk blocks per SM (0 = as many as fit)")
    ap.add_argument("--group", type=int, default=1,
                    help="lanes voting together (1, 2, 4, 8 or 32; 0 = split walk, "
                         "64 = interaction lists, 65 = one lane per particle over "
                         "sibling-ordered node records)")
    ap.add_argument("--no-kahan", action="store_true", help="plain FP32 force sums")
    ap.add_argument("--static-share", type=int, default=90)
    ap.add_argument("--no-graph", action="store_true", help="launch each step's kernels directly")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-theta07", action="store_true",
                    help="skip the headline workload at theta 0.7")
    ap.add_argument("--no-served", action="store_true")
    ap.add_argument("--no-large", action="store_true")
    ap.add_argument("--no-large-errors", dest="large_errors", action="store_false",
                    help="skip the large leg's oracle check (an FP64 tree of 2^24 particles)")
    ap.add_argument("--forest-systems", type=int, default=512)
    ap.add_argument("--forest-steps", type=int, default=100)
    ap.add_argument("--plain-steps", type=int, default=10)
    ap.add_argument("--serve-light-seconds", type=float, default=8.0,
                    help="seconds of arrivals for the half-load served run (0 = skip)")
    ap.add_argument("--serve-budget-gb", type=float, default=160.0,
                    help="HBM budget of each rank's server (GB)")
    ap.add_argument("--serve-seconds", type=float, default=0.5,
                    help="length of the Poisson arrival window (200 requests/s)")
    ap.add_argument("--workload", default="uniform1m", choices=sorted(WORKLOADS))
    ap.add_argument("--theta", type=float, default=None,
                    help="opening angle of the main leg (default: the workload's)")
    args = ap.parse_args()
    globals().update(WORKLOADS[args.workload])
    if args.theta is not None:
        globals()["THETA"] = args.theta
        globals()["WORKLOAD"] = WORKLOAD.replace("theta=0.5", f"theta={args.theta}")
    if args.warmup < 3 and args.impl != "reference":
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
