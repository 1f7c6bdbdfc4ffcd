"""Benchmark: SPH particle-updates/s of the leapfrog step on one GB300.

Workload: 3D Sedov-Taylor blast, 128^3 = 2,097,152 particles on a jittered
lattice (the seeded generator in paper_1909_07439_gb300.inputs).  One bench
step is one full sph_step: kick/drift, Morton-key tree build (keys, radix
sort, permutation, chop), group walk + h-rho Newton density solve, force
pass, closing kick and Courant step, all on the device.

Prints ONE JSON line (rank 0).  ``--impl reference`` times the FP64 CPU
oracle on a bounded sample of the same workload instead (the CPU baseline
arm).  Multi-GPU runs are independent replicas (the step is a single problem
and is not sharded), launched one process per GPU by torchrun.
"""
from __future__ import annotations

import argparse
import csv
import io
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "SPH particle-updates/s & pair-interactions/s (1 GB300); batched/adjoint vs plain"
UNIT = "particle-updates/s"
SIDE = 128
# Algorithmic FP32 operations per pair, counted on the oracle's operation
# list (the plain definition, Eqs. 1-15, as oracle/sph_oracle.c writes it:
# FMA = 2, add / sub / mul / div = 1, sqrt not counted):
#  force pair in the force set (orc_force): separation 3, r^2 5, 2 h_max 1,
#  v_ij . rhat 9 (with the divide), signal speed 3, F(r, h_i) 10 and
#  F(r, h_j) 10 (q = r/h, f'(q) 4, C f' / h^4 5), P_j 3, c_j 2, coefficient
#  12, acceleration 9, pressure work 3, conduction speed 4, conduction 12 = 86;
#  the viscous terms of approaching pairs (q^i, q^j, heating: 21 more) are
#  not counted, so 86 is a lower bound.
#  density sweep pair (density_sums): separation 3, r^2 5, W 12, dW/dh 21,
#  the two sums 4 = 45.
#  neighbour-list candidate test: canonical squared distance 3 sub 3 mul 2 add = 8.
FLOP_FORCE_PAIR = 86
FLOP_DENSITY_PAIR = 45
FLOP_TEST = 8
# The same counts for the other kernels: the branch-free shape functions cost
# more than M4's (f: M4 6, M6 16, Wendland C6 12; f': M4 4, M6 14, Wendland
# C6 13 operations), and a force pair evaluates f' twice, a density pair f
# twice (W and dW/dh) and f' once.
FLOP_PAIR = {0: (FLOP_FORCE_PAIR, FLOP_DENSITY_PAIR), 1: (106, 75), 2: (104, 66)}
# Executed FP32 operations per force pair of the list kernel
# (2 FFMA + FADD + FMUL from ncu's sass instruction counters over one launch
# of the 128^3 step, 2.71e9 FFMA, 2.05e9 FADD, 3.54e9 FMUL, divided by that
# launch's 1.3107e8 pairs; the count includes the list entries outside the
# pair set, which the kernel evaluates with zero mass).
EXEC_FLOP_FORCE_PAIR = 84.0
# DRAM bytes (read + write) per launch of the pair kernels from one ncu capture
# of the 128^3 step; None where the kernel changed after the capture.
NCU_TRAFFIC = {"nlist_kernel": 135.070208e6 + 602.764288e6,
               "density_list_kernel": 918.412544e6 + 34.043392e6,
               "force_list_kernel": 1.00118e9 + 29.120512e6}
# Issue slots busy (smsp__issue_active, fraction of the active cycles) in the
# same ncu captures: the list build is bound by instruction issue, which its
# FP32 fraction (8 FLOP per candidate test) does not show.
NCU_ISSUE_ACTIVE = {"nlist_kernel": 0.756, "density_list_kernel": 0.682, "force_list_kernel": 0.656}
# Self-gravity FP32 operations per interaction (softened pair: separation 3,
# r^2 + eps^2 6, the inverse powers 3, m/r and m/r^3 2, acceleration 6,
# potential 1 = 21; quadrupole cell: the same 20 plus Q d 15, d.Q.d 5, the
# cell terms 20 = 60; the reciprocal square root counted as one operation).
FLOP_GRAV_PART = 21
FLOP_GRAV_CELL = 60
# Algorithmic bytes per particle of the tree build (bbox 20, keys 28, four
# 12-byte-key passes of the sort read and written 96, run fix-up 8, gather of
# pos, vel, half-step vel, h and perm read and written 112 plus the 32-byte
# record and 8-byte key 40, chop and node bounds 28).
TREE_BYTES_PER_PARTICLE = 332


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int, interval_ms: int = 20):
        self.dev = device_index
        self.interval = interval_ms
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", str(self.interval)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        rows = [r for r in csv.reader(io.StringIO(out)) if len(r) >= 9]
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except ValueError:
                continue
            for k, name in enumerate(names):
                if r[5 + k].strip().lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(mx)) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measure_fp32_peak(native, torch, sms, device_index, target_ms=400.0):
    """Measured FP32 peak: the library's multiply-add chain probe (scalar FMA
    and packed FP32x2 FMA), 8 blocks of 256 threads per SM, timed with CUDA
    events on the launching stream while nvidia-smi samples the SM clock.
    Returns TFLOP/s of each form and the median SM clock under the probe."""
    sink = torch.zeros(1, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    blocks = 8 * sms
    out = {}
    clocks = ClockSampler(device_index, interval_ms=20)
    for packed in (False, True):
        flop_per_iter = blocks * 256 * (32 if packed else 16)
        iters = 256
        for _ in range(2):                       # warm-up, then size the run
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            native.sph_fp32_probe(sink, blocks, iters, packed)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            iters = max(256, int(iters * target_ms / max(ms, 1e-3)))
        if packed is False:
            clocks.start()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        native.sph_fp32_probe(sink, blocks, iters, packed)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        out["ffma2" if packed else "ffma"] = flop_per_iter * iters / (ms / 1e3) / 1e12
    clk = clocks.stop()
    out["sm_mhz"] = clk.get("sm_mhz")
    out["clock_samples"] = clk.get("samples")
    out["reasons"] = clk.get("reasons")
    return out


def roofline(stage_ms, stats, reps, fp32_peak, peak_basis, hbm_peak, n, kernel=0):
    """Roofline of the pair-kernel stages (FP32 ALU bound) and of the tree
    build (HBM bound), from the library's stage timers (CUDA events on the
    launching stream) summed over `reps` launches and the work counters."""
    f_force, f_dens = FLOP_PAIR[kernel]
    work = {"lists": ("nlist_kernel", stats["density_candidates"] * FLOP_TEST, None),
            "density": ("density_list_kernel", stats["density_pairs"] * f_dens, None),
            "force": ("force_list_kernel", stats["force_pairs"] * f_force,
                      stats["force_pairs"] * EXEC_FLOP_FORCE_PAIR if kernel == 0 else None)}
    stages = {}
    for st, (kern, flop, exe) in work.items():
        ms = stage_ms[st] / reps
        if ms <= 0:
            continue
        ach = flop / reps / (ms / 1e3) / 1e12
        stages[st] = {"kernel": kern, "launch_ms": round(ms, 4), "achieved": round(ach, 3),
                      "frac": round(ach / fp32_peak, 4), "issue_active_ncu": NCU_ISSUE_ACTIVE.get(kern)}
        if exe is not None:
            stages[st]["achieved_executed"] = round(exe / reps / (ms / 1e3) / 1e12, 3)
    dom = max(stages, key=lambda k: stages[k]["launch_ms"])
    d = stages[dom]
    roof = {"kernel": d["kernel"], "bound": "alu", "achieved": d["achieved"],
            "peak": round(fp32_peak, 2), "unit": "TFLOP/s", "frac": d["frac"],
            "traffic": NCU_TRAFFIC.get(d["kernel"]), "issue_active_ncu": NCU_ISSUE_ACTIVE.get(d["kernel"]),
            "peak_basis": peak_basis,
            "launch_ms": d["launch_ms"], "flop_per_pair": f_force if dom == "force" else None,
            "stages": stages}
    if "achieved_executed" in d:
        roof["achieved_executed"] = d["achieved_executed"]
        roof["frac_executed"] = round(d["achieved_executed"] / fp32_peak, 4)
    tree_ms = stage_ms["tree"] / reps
    if tree_ms > 0:
        gbs = TREE_BYTES_PER_PARTICLE * n / (tree_ms / 1e3) / 1e9
        roof["tree_build"] = {"bound": "hbm", "achieved": round(gbs, 1), "peak": hbm_peak,
                              "unit": "GB/s", "frac": round(gbs / hbm_peak, 4),
                              "bytes_per_particle": TREE_BYTES_PER_PARTICLE,
                              "launch_ms": round(tree_ms, 4)}
    return roof


def shard_instances(sizes, world_size):
    """Split independent instances over ranks, balancing particle counts
    (largest first onto the least-loaded rank); deterministic."""
    load = [0] * world_size
    parts = [[] for _ in range(world_size)]
    for k in sorted(range(len(sizes)), key=lambda k: (-int(sizes[k]), k)):
        r = min(range(world_size), key=lambda q: (load[q], q))
        parts[r].append(k)
        load[r] += int(sizes[k])
    return [sorted(p) for p in parts]


def aggregate(local_ms, units, world_size, all_reduce_max=None):
    """Whole-job rate: units processed by all ranks over the slowest rank's time."""
    ms = all_reduce_max(local_ms) if (all_reduce_max and world_size > 1) else local_ms
    return units * world_size / (ms / 1e3), ms


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ----------------------------------------------------------------- our arm
def run_ours(args):
    import torch
    from paper_1909_07439_gb300 import DeviceState, build, inputs, native

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    build.build()
    native.load()
    w = inputs.sedov_lattice(args.side)
    n = w.n
    ctx = native.sph_create(n, local)
    s = DeviceState.from_arrays(w.pos, w.vel, w.h, device=f"cuda:{local}")
    p = native.sph_params_default()
    if args.n_leaf:
        p.n_leaf = args.n_leaf
    if args.n_group:
        p.n_group = args.n_group
    if args.tile:
        p.tile = args.tile
    if args.pair_shape:
        p.pair_targets, p.pair_warps, p.pair_unroll = (int(x) for x in args.pair_shape.split(","))
    stream = torch.cuda.current_stream()
    d_dt = torch.zeros(1, dtype=torch.float32, device="cuda")
    d_t = torch.zeros(1, dtype=torch.float64, device="cuda")
    # initial evaluation (untimed): tree, density, force, Courant step
    native.sph_build_tree(ctx, s.c, p)
    native.sph_density(ctx, s.c, p)
    native.sph_force(ctx, s.c, p)
    native.sph_timestep(ctx, s.c, p, d_dt)
    native.sph_sync(ctx)
    for _ in range(args.warmup):
        native.sph_step(ctx, s.c, p, d_dt, d_t)
    native.sph_sync(ctx)
    tuned = None
    if not (args.n_leaf or args.n_group):
        # N_group and N_leaf tuned on the warmed-up state (untimed, state restored)
        from paper_1909_07439_gb300 import autotune
        p, tuned = autotune.tune_step(ctx, s, d_dt, f"sedov{args.side}", base=p, steps=20)
        for _ in range(2):
            native.sph_step(ctx, s.c, p, d_dt, d_t)
        native.sph_sync(ctx)
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    fp32 = measure_fp32_peak(native, torch, sms, local)
    native.sph_get_stats(ctx)          # reset counters
    native.sph_get_timing(ctx)         # reset stage timers
    native.sph_set_timing(ctx, True)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")  # > 129 MB L2
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    clocks = ClockSampler(local, interval_ms=10)
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.05)                   # the sampler's first sample lands in the region
    for k in range(args.steps):
        flush.zero_()                  # L2 flushed between timed steps (outside the events)
        evs[k][0].record(stream)
        native.sph_step(ctx, s.c, p, d_dt, d_t)
        evs[k][1].record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    if ws > 1:
        torch.distributed.barrier()
    native.sph_sync(ctx)
    step_ms = [a.elapsed_time(b) for a, b in evs]
    total_ms = float(sum(step_ms))
    stage_ms, launches = native.sph_get_timing(ctx)
    native.sph_set_timing(ctx, False)
    stats = native.sph_get_stats(ctx)
    def _max(x):
        t = torch.tensor([x], device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        return float(t.item())

    value, total_ms = aggregate(total_ms, n * args.steps, ws, _max)
    pairs = stats["density_pairs"] + stats["force_pairs"]
    pair_rate = pairs * ws / (total_ms / 1e3)

    # roofline: the longest pair-kernel stage against the measured FP32 peak,
    # the tree build against the measured HBM copy bandwidth
    pk, pk_kind = peaks()
    fp32_peak = max(fp32["ffma"], fp32["ffma2"])
    basis = (f"measured: FP32 multiply-add chain probe, {8 * sms} blocks of 256 threads, "
             f"scalar FMA {fp32['ffma']:.1f} and packed FP32x2 FMA {fp32['ffma2']:.1f} TFLOP/s at "
             f"median SM clock {fp32['sm_mhz']} MHz (nominal 2 x 128 lanes x {sms} SMs x "
             f"{pk.get('sm_max_mhz', 2070.0)} MHz = "
             f"{2 * 128 * sms * pk.get('sm_max_mhz', 2070.0) / 1e6:.2f})")
    roof = roofline(stage_ms, stats, args.steps, fp32_peak, basis, pk.get("hbm_gbs", 6800.0), n)
    roof["hbm_peak_basis"] = f"hbm_gbs of MEASURED_PEAKS.json ({pk_kind})"
    hold = clock_hold(native, ctx, s, p, d_dt, local) if rank == 0 else None
    clk["after_region"] = hold

    e2e = run_e2e(native, ctx, s, p, n, args, stream) if rank == 0 and not args.skip_e2e else None
    native.sph_destroy(ctx)
    del s
    batched = run_batched(args) if rank == 0 and args.batch_instances > 0 else None
    adjoint = run_adjoint(args) if rank == 0 and args.adjoint_side > 0 else None
    plummer = (run_plummer(args, fp32_peak, basis, pk.get("hbm_gbs", 6800.0))
               if rank == 0 and args.plummer_log2 > 0 else None)
    tube = (run_tube(args, fp32_peak, basis, pk.get("hbm_gbs", 6800.0))
            if rank == 0 and args.tube_scale > 0 else None)
    block = run_block(args) if rank == 0 and args.block_levels > 0 else None
    out = None
    if rank == 0:
        cpu = run_cpu_baseline(w, args.cpu_seconds) if args.cpu_seconds > 0 else None
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded Sedov lattice; no dataset)",
            "config": {"workload": f"sedov_blast_lattice_{args.side}^3", "n_particles": n,
                       "step": "sph_step: KDK + tree build + density Newton + force + Courant dt",
                       "kernel": "M4", "n_leaf": p.n_leaf, "n_group": p.n_group,
                       "tuned": tuned is not None,
                       "hfact": round(p.hfact, 4), "l2": "flushed between timed steps",
                       "parallelism": f"replicas x{ws}"},
            "pair_interactions_per_s": pair_rate,
            "autotune": tuned,
            "clocks": clk,
            "e2e": e2e,
            "gpu_launches": int(sum(launches.values())),
            "roofline": roof,
            "cpu_baseline": cpu,
            "stage_ms_per_step": {k: round(v / args.steps, 4) for k, v in stage_ms.items()},
            "work_per_step": {k: v / args.steps for k, v in stats.items()
                              if k not in ("n_nodes", "n_groups")},
            "tree": {"n_nodes": stats["n_nodes"], "n_groups": stats["n_groups"]},
            "sim_time": float(d_t.item()),
            "batched": batched,
            "adjoint": adjoint,
            "plummer": plummer,
            "tube": tube,
            "block": block,
        }
    if ws > 1:
        torch.distributed.destroy_process_group()
    return out


def clock_hold(native, ctx, s, p, d_dt, device_index, seconds=0.6):
    """SM clocks while the same step runs back to back for `seconds` right
    after the timed region (the timed region itself holds few samples).  The
    state and dt are restored afterwards, so later legs see the timed state."""
    import torch
    saved = {f: getattr(s, f).clone() for f in s.FIELDS4 + s.FIELDS1 + ("perm", "keys")}
    dt0 = d_dt.clone()
    c = ClockSampler(device_index, interval_ms=10)
    c.start()
    t0 = time.perf_counter()
    k = 0
    while time.perf_counter() - t0 < seconds:
        for _ in range(20):
            native.sph_step(ctx, s.c, p, d_dt)
        torch.cuda.synchronize()
        k += 20
    out = c.stop()
    out["steps"] = k
    for f, v in saved.items():
        getattr(s, f).copy_(v)
    d_dt.copy_(dt0)
    torch.cuda.synchronize()
    return out


def run_batched(args):
    """512 independent Sedov blasts (log-uniform sizes in [4096, 262144]),
    20 steps each with per-instance dt: one batched state, graph-replayed
    steps with persistent list and pair kernels, autotuned N_group and N_leaf; compared
    with the same instances advanced one after another by sph_step."""
    import torch
    from paper_1909_07439_gb300 import DeviceState, autotune, inputs, native
    ws, rank, _ = dist_env()
    sides = inputs.batch_sizes(args.batch_instances, seed=4)
    mine = shard_instances(sides ** 3, ws)[rank]   # this rank's instances, no exchange
    w, off = inputs.sedov_batch(args.batch_instances, seed=4, only=mine)
    k = len(off) - 1
    ctx = native.sph_create(w.n, 0)
    s = DeviceState.from_arrays(w.pos, w.vel, w.h)
    d_off = torch.as_tensor(off, device="cuda")
    dt = torch.zeros(k, dtype=torch.float32, device="cuda")
    t = torch.zeros(k, dtype=torch.float64, device="cuda")
    p, report = autotune.tune_batch(ctx, s, d_off, k)
    native.sph_batch_evaluate(ctx, s.c, d_off, k, p, dt)
    native.sph_batch_step(ctx, s.c, d_off, k, 1, p, dt, t)      # records the graph
    native.sph_sync(ctx)
    native.sph_get_stats(ctx)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    native.sph_batch_step(ctx, s.c, d_off, k, args.batch_steps, p, dt, t)
    e1.record()
    torch.cuda.synchronize()
    native.sph_sync(ctx)
    t_batch = e0.elapsed_time(e1) / 1e3
    stats = native.sph_get_stats(ctx)
    native.sph_destroy(ctx)
    del s
    # the same instances one after another through the single-instance path,
    # with the batch's tuned parameters and with the single-instance step's
    # (N_group = N_leaf = 16, 16 targets per batch, 4 warps, 2 entries): the
    # faster of the two is the baseline
    nmax = int(np.max(np.diff(off)))
    ctx = native.sph_create(nmax, 0)
    seq = {}
    for name, p1 in (("batch_params", native.sph_params_default(
                         n_group=p.n_group, n_leaf=p.n_leaf, pair_targets=p.pair_targets,
                         pair_warps=p.pair_warps, pair_unroll=p.pair_unroll)),
                     ("plain_params", native.sph_params_default(
                         n_group=16, n_leaf=16, pair_targets=16, pair_warps=4, pair_unroll=2))):
        states = []
        for i in range(k):
            a, b = int(off[i]), int(off[i + 1])
            si = DeviceState.from_arrays(w.pos[a:b], w.vel[a:b], w.h[a:b])
            di = torch.zeros(1, dtype=torch.float32, device="cuda")
            native.sph_build_tree(ctx, si.c, p1)
            native.sph_density(ctx, si.c, p1)
            native.sph_force(ctx, si.c, p1)
            native.sph_timestep(ctx, si.c, p1, di)
            native.sph_step(ctx, si.c, p1, di)
            states.append((si, di))
        native.sph_sync(ctx)
        torch.cuda.synchronize()
        e0.record()
        for si, di in states:
            for _ in range(args.batch_steps):
                native.sph_step(ctx, si.c, p1, di)
        e1.record()
        torch.cuda.synchronize()
        native.sph_sync(ctx)
        seq[name] = e0.elapsed_time(e1) / 1e3
        del states
    t_seq = min(seq.values())
    native.sph_destroy(ctx)
    updates = w.n * args.batch_steps
    return {"workload": f"{k} Sedov blasts, sizes log-uniform in [4096, 262144] (seeded), "
                        f"{w.n} particles", "steps": args.batch_steps,
            "value": updates / t_batch, "unit": UNIT,
            "plain_sequential_value": updates / t_seq, "batched_over_plain": t_seq / t_batch,
            "plain_sequential_ms": {k2: 1e3 * v / args.batch_steps for k2, v in seq.items()},
            "pair_interactions_per_s": (stats["density_pairs"] + stats["force_pairs"]) / t_batch,
            "autotune": report, "ms_per_step": 1e3 * t_batch / args.batch_steps}


def run_adjoint(args):
    """Differentiable form: 64^3 Sedov blast, 20-step rollout, loss = mean
    rho^2 of 1024 seeded probes, gradients w.r.t. initial v, u and alpha_AV
    with checkpoints every 5 steps; timed against the same rollout without
    gradients."""
    import torch
    from paper_1909_07439_gb300 import DeviceState, inputs, native
    w = inputs.sedov_lattice(args.adjoint_side)
    probes = torch.as_tensor(inputs.probe_indices(w.n, 1024), device="cuda")
    ctx = native.sph_create(w.n, 0)
    s = DeviceState.from_arrays(w.pos, w.vel, w.h)
    p = native.sph_params_default()
    g = torch.zeros((w.n, 4), dtype=torch.float32, device="cuda")
    native.sph_rollout(ctx, s.c, p, 20, 5, probes, 1024, g)       # allocates the work buffers
    t0 = time.perf_counter()
    loss_f, _ = native.sph_rollout(ctx, s.c, p, 20, 5, probes, 1024)
    t1 = time.perf_counter()
    loss_b, ga = native.sph_rollout(ctx, s.c, p, 20, 5, probes, 1024, g)
    t2 = time.perf_counter()
    native.sph_destroy(ctx)
    n_upd = w.n * 20
    return {"workload": f"Sedov lattice {args.adjoint_side}^3 ({w.n} particles), 20 KDK steps, "
                        f"1024 probes, checkpoints every 5", "loss": loss_f,
            "forward_value": n_upd / (t1 - t0), "forward_backward_value": n_upd / (t2 - t1),
            "unit": UNIT, "adjoint_over_forward_time": (t2 - t1) / (t1 - t0),
            "grad_norm_v": float(torch.linalg.vector_norm(g[:, :3])),
            "grad_norm_u": float(torch.linalg.vector_norm(g[:, 3])), "dL_dalpha": ga}


def run_plummer(args, fp32_peak, basis, hbm_peak):
    """Strongly inhomogeneous evaluation: 2^24-particle Plummer sphere,
    tree build + density + force of one evaluation, tree sizes and launch
    shape tuned on the state; roofline of its stages and the oracle timed on
    a sample of the same workload."""
    import torch
    from paper_1909_07439_gb300 import DeviceState, inputs, native
    from paper_1909_07439_gb300 import autotune
    w = inputs.plummer(1 << args.plummer_log2)
    ctx = native.sph_create(w.n, 0)
    s = DeviceState.from_arrays(w.pos, w.vel, w.h)
    p = native.sph_params_default()
    native.sph_build_tree(ctx, s.c, p)
    native.sph_density(ctx, s.c, p)      # converges h from the analytic-density guess
    native.sph_force(ctx, s.c, p)
    native.sph_sync(ctx)
    d_dt = torch.zeros(1, dtype=torch.float32, device="cuda")
    p, tuned = autotune.tune_step(ctx, s, d_dt, f"plummer{args.plummer_log2}", base=p, steps=2,
                                  evaluate_only=True,
                                  candidates=[(g, l) for g in (8, 16, 32) for l in (16, 32, 64)])
    native.sph_get_stats(ctx)
    native.sph_get_timing(ctx)
    native.sph_set_timing(ctx, True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 3
    e0.record()
    for _ in range(reps):
        native.sph_build_tree(ctx, s.c, p)
        native.sph_density(ctx, s.c, p)
        native.sph_force(ctx, s.c, p)
    e1.record()
    torch.cuda.synchronize()
    native.sph_sync(ctx)
    ms = e0.elapsed_time(e1) / reps
    stage, _ = native.sph_get_timing(ctx)
    stats = native.sph_get_stats(ctx)
    grav = run_gravity(native, ctx, s, w, fp32_peak)
    native.sph_destroy(ctx)
    hh = s.numpy("h")
    roof = roofline(stage, stats, reps, fp32_peak, basis, hbm_peak, w.n)
    cpu = run_cpu_baseline(w, args.cpu_seconds) if args.cpu_seconds > 0 else None
    return {"workload": f"Plummer sphere a = 0.1 truncated at r = 1, {w.n} particles",
            "roofline": roof, "cpu_baseline": cpu,
            "ms_per_evaluation": ms, "value": w.n / (ms / 1e3), "unit": UNIT,
            "pair_interactions_per_s": (stats["density_pairs"] + stats["force_pairs"]) / reps / (ms / 1e3),
            "stage_ms": {k: v / reps for k, v in stage.items()},
            "h_range": [float(hh.min()), float(hh.max())],
            "streamed_groups": stats["streamed_groups"] / reps,
            "n_nodes": stats["n_nodes"], "n_groups": stats["n_groups"],
            "n_group": p.n_group, "n_leaf": p.n_leaf, "autotune": tuned, "gravity": grav}


def run_gravity(native, ctx, s, w, fp32_peak, theta=0.5, eps=0.01):
    """Self-gravity (Barnes-Hut, quadrupole cells) on the built tree of the
    Plummer state: moments pass + walk, timed with CUDA events, for groups of
    16 and 32 particles (the faster one reported, both listed)."""
    import torch
    out = torch.zeros((w.n, 4), dtype=torch.float32, device="cuda")
    trials = []
    for ng in (16, 32):
        p = native.sph_params_default(grav_G=1.0, grav_eps=eps, grav_theta=theta, n_group=ng)
        native.sph_build_tree(ctx, s.c, p)
        native.sph_gravity(ctx, s.c, p, out)          # warm-up
        native.sph_sync(ctx)
        native.sph_get_stats(ctx)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 3
        e0.record()
        for _ in range(reps):
            native.sph_gravity(ctx, s.c, p, out)
        e1.record()
        torch.cuda.synchronize()
        native.sph_sync(ctx)
        st = native.sph_get_stats(ctx)
        trials.append((e0.elapsed_time(e1) / reps, ng, st["gravity_cells"] / reps,
                       st["gravity_particles"] / reps))
    ms, ng, cells, parts = min(trials)
    flop = cells * FLOP_GRAV_CELL + parts * FLOP_GRAV_PART
    ach = flop / (ms / 1e3) / 1e12
    return {"theta": theta, "eps": eps, "n_group": ng, "ms_per_evaluation": ms,
            "trials": [{"n_group": t[1], "ms": t[0], "interactions_per_particle": (t[2] + t[3]) / w.n}
                       for t in trials],
            "value": w.n / (ms / 1e3), "unit": "particle gravity evaluations/s",
            "interactions_per_particle": (cells + parts) / w.n,
            "interactions_per_s": (cells + parts) / (ms / 1e3),
            "roofline": {"bound": "alu", "achieved": round(ach, 3), "peak": round(fp32_peak, 2),
                         "unit": "TFLOP/s", "frac": round(ach / fp32_peak, 4),
                         "flop_per_interaction": {"cell": FLOP_GRAV_CELL, "particle": FLOP_GRAV_PART}}}


def run_tube(args, fp32_peak, basis, hbm_peak):
    """Sod shock tube (Sect. 4.1) with the M6 kernel and periodic boundaries,
    the paper's setup scaled by --tube-scale per axis: untimed steps until
    the waves have formed, then timed steps with CUDA events."""
    import torch
    from paper_1909_07439_gb300 import DeviceState, inputs, native
    k = args.tube_scale
    w = inputs.sod_tube(256 * k, 24 * k)
    m = w.meta
    ctx = native.sph_create(w.n, 0)
    s = DeviceState.from_arrays(w.pos, w.vel, w.h)
    p = native.sph_params_default(kernel=1, hfact=1.0, gamma=m["gamma"], box_lo=m["box_lo"],
                                  box_len=m["box_len"], n_group=16)
    d_dt = torch.zeros(1, dtype=torch.float32, device="cuda")
    d_t = torch.zeros(1, dtype=torch.float64, device="cuda")
    native.sph_build_tree(ctx, s.c, p)
    native.sph_density(ctx, s.c, p)
    native.sph_force(ctx, s.c, p)
    native.sph_timestep(ctx, s.c, p, d_dt)
    for _ in range(30):
        native.sph_step(ctx, s.c, p, d_dt, d_t)
    native.sph_sync(ctx)
    # tree sizes and launch shape tuned on this state (untimed, state restored)
    from paper_1909_07439_gb300 import autotune
    p, tuned = autotune.tune_step(ctx, s, d_dt, f"sod_m6_{k}", base=p, steps=2)
    native.sph_get_stats(ctx)
    native.sph_get_timing(ctx)
    native.sph_set_timing(ctx, True)
    reps = 40
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(reps):
        native.sph_step(ctx, s.c, p, d_dt, d_t)
    e1.record()
    torch.cuda.synchronize()
    native.sph_sync(ctx)
    ms = e0.elapsed_time(e1) / reps
    stage, _ = native.sph_get_timing(ctx)
    native.sph_set_timing(ctx, False)
    stats = native.sph_get_stats(ctx)
    t = d_t.item()
    native.sph_destroy(ctx)
    roof = roofline(stage, stats, reps, fp32_peak, basis, hbm_peak, w.n, kernel=1)
    return {"workload": f"Sod shock tube, M6 kernel, periodic box, {256 * k}x{24 * k}^2 | "
                        f"{128 * k}x{12 * k}^2 particles ({w.n})",
            "value": w.n / (ms / 1e3), "unit": UNIT, "ms_per_step": ms, "steps": reps,
            "sim_time_after": t,
            "pair_interactions_per_s": (stats["density_pairs"] + stats["force_pairs"]) / reps / (ms / 1e3),
            "stage_ms": {kk: v / reps for kk, v in stage.items()},
            "work_per_step": {kk: v / reps for kk, v in stats.items()
                              if kk in ("density_pairs", "force_pairs", "newton_iters",
                                        "density_rewalks", "force_rewalks", "list_overflows")},
            "autotune": tuned, "roofline": roof}


def run_block(args):
    """Block (individual) time steps on the Sedov blast: from the state after
    20 global steps, the same span of time as one block of 2^L substeps of
    the Courant dt_min, taken (a) as 2^L global steps of dt_min and (b) as one
    block step with each particle on its own level; both timed with CUDA
    events from the same saved state."""
    import torch
    from paper_1909_07439_gb300 import DeviceState, inputs, native
    L = args.block_levels
    w = inputs.sedov_lattice(args.side)
    ctx = native.sph_create(w.n, 0)
    s = DeviceState.from_arrays(w.pos, w.vel, w.h)
    p = native.sph_params_default(n_group=16)
    d_dt = torch.zeros(1, dtype=torch.float32, device="cuda")
    native.sph_build_tree(ctx, s.c, p)
    native.sph_density(ctx, s.c, p)
    native.sph_force(ctx, s.c, p)
    native.sph_timestep(ctx, s.c, p, d_dt)
    for _ in range(20):
        native.sph_step(ctx, s.c, p, d_dt)
    native.sph_sync(ctx)
    saved = {f: getattr(s, f).clone() for f in s.FIELDS4 + s.FIELDS1 + ("perm", "keys")}
    d_level = torch.zeros(w.n, dtype=torch.int32, device="cuda")
    native.sph_block_levels(ctx, s.c, p, L, d_dt, d_level)
    native.sph_sync(ctx)
    dt0 = d_dt.item()
    levels = np.bincount(d_level.cpu().numpy(), minlength=L + 1).tolist()

    def restore():
        for f, t in saved.items():
            getattr(s, f).copy_(t)
        torch.cuda.synchronize()

    out = {}
    for mode in ("global", "block"):
        best = None
        for rep in range(3):
            restore()
            native.sph_get_stats(ctx)
            native.sph_get_timing(ctx)
            native.sph_set_timing(ctx, True)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            if mode == "global":
                for _ in range(1 << L):
                    d_dt.fill_(dt0)
                    native.sph_step(ctx, s.c, p, d_dt)
            else:
                d_dt.fill_(dt0)
                native.sph_step_block(ctx, s.c, p, L, d_level, d_dt)
            e1.record()
            torch.cuda.synchronize()
            native.sph_sync(ctx)
            st = native.sph_get_stats(ctx)
            stage, _ = native.sph_get_timing(ctx)
            native.sph_set_timing(ctx, False)
            ms = e0.elapsed_time(e1)
            if best is None or ms < best[0]:
                best = (ms, st["force_pairs"], st["density_pairs"], stage)
        out[mode] = {"ms": best[0], "force_pairs": best[1], "density_pairs": best[2],
                     "stage_ms": {k: round(v, 4) for k, v in best[3].items()}}
    native.sph_destroy(ctx)
    span = (1 << L) * dt0
    return {"workload": f"Sedov lattice {args.side}^3 after 20 steps, {1 << L} x dt_min "
                        f"({span:.3e} of simulated time)",
            "levels": levels, "global_ms": out["global"]["ms"], "block_ms": out["block"]["ms"],
            "speedup": out["global"]["ms"] / out["block"]["ms"],
            "force_pairs": {"global": out["global"]["force_pairs"], "block": out["block"]["force_pairs"]},
            "stage_ms": {"global": out["global"]["stage_ms"], "block": out["block"]["stage_ms"]},
            "value": w.n * (1 << L) / (out["block"]["ms"] / 1e3),
            "unit": "particle-updates/s at dt_min resolution (block steps)"}


def run_e2e(native, ctx, s, p, n, args, stream):
    """Same metric through the C ABI with the state in pinned HOST memory:
    every step copies the inputs in and the whole state back."""
    import ctypes
    import torch
    host = {k: getattr(s, k)[:n].cpu().pin_memory() for k in s.FIELDS4 + s.FIELDS1 + ("perm", "keys")}
    hs = native.sph_state()
    hs.n = n
    for k, t in host.items():
        setattr(hs, k, t.data_ptr())
    dt = ctypes.c_float(1e-6)
    d = torch.zeros(1, dtype=torch.float32, device="cuda")
    native.sph_timestep(ctx, s.c, p, d)
    dt.value = d.item()
    native.sph_step_host(ctx, hs, p, 1, dt)  # first call allocates the mirror
    k = max(1, min(args.steps, 10))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(k):
        native.sph_step_host(ctx, hs, p, 1, dt)
    t1 = time.perf_counter()
    h2d = n * (16 * 3 + 4 + 4) + 4
    d2h = n * (16 * 3 + 4 * 5 + 4 + 8) + 4
    return {"value": n * k / (t1 - t0), "unit": UNIT, "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h, "steps": k,
            "note": "sph_step_host: pinned host state, H2D + step + D2H inside the timed region"}


# ------------------------------------------------------------ CPU baseline
def oracle_sample_rate(w, target_seconds, seed=12345):
    """Time the FP64 oracle's per-particle work on a sample of targets:
    the h-rho solve (brute force over all n) plus the force pass (brute force
    over all n).  The force leg uses the generator's h and unit rho, Omega for
    the non-sampled particles; its cost is the O(n) pair scan per target."""
    import oracle
    oracle.build()
    x = w.pos[:, :3].astype(np.float64)
    v = w.vel[:, :3].astype(np.float64)
    m = w.pos[:, 3].astype(np.float64)
    u = w.vel[:, 3].astype(np.float64)
    h0 = w.h.astype(np.float64)
    rng = np.random.default_rng(seed)

    def run(k):
        t = np.sort(rng.choice(w.n, size=k, replace=False))
        t0 = time.perf_counter()
        d = oracle.density(x, v, m, h0, targets=t)
        hh, rr, oo = h0.copy(), np.ones(w.n), np.ones(w.n)
        hh[t], rr[t], oo[t] = d.h, d.rho, d.omega
        oracle.force(x, v, m, u, hh, rr, oo, targets=t)
        return time.perf_counter() - t0

    k = 16
    dt = run(k)
    while dt < 0.5 and k < 1 << 16:
        k *= 2
        dt = run(k)
    k = max(1, int(k * target_seconds / max(dt, 1e-9)))
    dt = run(k)
    return k, dt


def run_cpu_baseline(w, seconds):
    k, dt = oracle_sample_rate(w, seconds)
    return {"value": k / dt, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"{k} seeded target particles of the {w.n}-particle workload: FP64 h-rho "
                      f"Newton solve + force, each brute force over all {w.n} particles "
                      f"({dt:.1f} s)"}


def run_reference(args):
    ws, rank, local = dist_env()
    if rank != 0:
        return None
    from paper_1909_07439_gb300 import inputs
    w = inputs.sedov_lattice(args.side)
    per_step = max(1.0, min(10.0, 120.0 / max(1, args.steps + args.warmup)))
    for _ in range(args.warmup):
        oracle_sample_rate(w, per_step / 4)
    total_k, total_t = 0, 0.0
    for _ in range(args.steps):
        k, dt = oracle_sample_rate(w, per_step)
        total_k += k
        total_t += dt
    value = total_k / total_t
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * total_t / args.steps,
            "ms_per_step_basis": "measured wall time of one sample step (a bounded sample of "
                                 "target particles, not the whole workload)",
            "extrapolated_ms_per_full_step": 1e3 * w.n / value,
            "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded Sedov lattice)",
            "config": {"workload": f"sedov_blast_lattice_{args.side}^3", "n_particles": w.n},
            "cpu_baseline": {"kind": "oracle", "cores": os.cpu_count(), "value": value,
                             "unit": UNIT,
                             "sample": f"{total_k} target particles over {args.steps} steps, "
                                       f"each brute force over all {w.n} particles"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "note": "FP64 brute-force CPU oracle (the reference arm); per-particle rate"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--side", type=int, default=SIDE)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--skip-e2e", action="store_true", help="profiling runs: no host-buffer leg")
    ap.add_argument("--n-leaf", type=int, default=0, help="override N_leaf (paper: 16)")
    ap.add_argument("--n-group", type=int, default=0, help="override N_group (paper: 8)")
    ap.add_argument("--tile", type=int, default=0, help="override the neighbour-list tile")
    ap.add_argument("--pair-shape", default="",
                    help="override the pair kernels' launch shape: targets,warps,unroll "
                         "(with --n-leaf/--n-group it replaces the autotuner's choice)")
    ap.add_argument("--batch-instances", type=int, default=512)
    ap.add_argument("--batch-steps", type=int, default=20)
    ap.add_argument("--adjoint-side", type=int, default=64)
    ap.add_argument("--plummer-log2", type=int, default=24)
    ap.add_argument("--block-levels", type=int, default=3,
                    help="block time step leg: levels below dt_min 2^L (0: skip)")
    ap.add_argument("--tube-scale", type=int, default=2,
                    help="Sod/M6/periodic leg: the paper's tube scaled per axis (0: skip)")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    out = run_reference(args) if args.impl == "reference" else run_ours(args)
    if out is not None:
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
