#!/usr/bin/env python
"""Throughput benchmark of the GB300 Kino-PAX+ planner (valid expansions/s).

A step is one planning run of the whole hot path on one synthetic problem:
kpx_reset + kpx_iterate(I) (I = the configuration's iteration count), i.e.
I passes of Propagate -> winner select -> UpdateTree append -> PruneNodes with
the active-set compaction.  Every step of a run is the same deterministic
problem, so each step does identical work.

Default workload: 12D quadcopter in a 1,000-box building (9 zig-zag walls
with 0.04 x 0.04 openings plus 964 clutter boxes), RK4 h = 0.005,
16^3 x 4^3 regions, tree cap 2^22, lambda = 128, 200 iterations.

Printed (rank 0, one JSON line): value = valid expansions/s over the timed
device region (inputs resident in HBM, L2 flushed between steps), e2e = the
same metric through the C ABI with host buffers (kpx_create from host arrays,
iterate, kpx_best_trajectory to host, destroy), the roofline of the dominant
kernel (propagate, bound by FP32/ALU issue), the roofline of the tree update
(mark + scan + append + prune, against HBM bandwidth), the FP64 oracle timed
on the host cores, and SM clocks sampled during the timed region.

--impl reference times the FP64 oracle (the CPU reference of this project) on
the same workload and prints the same line with "impl": "reference".
"""
from __future__ import annotations

import argparse
import ctypes
import json
import math
import os
import shutil
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2602_02846_gb300 import scenes  # noqa: E402

METRIC = "valid expansions/s"
UNIT = "valid expansions/s"

# Algorithmic FP32 work of one integration step (dynamics + integrator + cost
# + state/workspace checks; an FMA counts 2, sin/cos 1 each) and of one
# point-in-box test (6 comparisons).
OPS_PER_STEP = {scenes.DI6: 22.0, scenes.DUBINS6: 96.0, scenes.QUAD12: 270.0}
OPS_PER_BOX_TEST = 6.0
SM_COUNT_FALLBACK = 152
# DRAM bytes (read + write) of one propagate launch from the ncu captures in
# profiles/ (the kernel build named there); None for a workload not captured.
FUSED_DRAM_BYTES = {
    "dubins6_forest300": 195072,     # profiles/k_fused_dubins6_forest300.md (the timed step's graph launch)
}
PROPAGATE_DRAM_BYTES = {
    "quad12_building1000": 6868736,  # profiles/k_propagate_quad12_building1000.md (iteration 100)
}
FP32_LANES_PER_SM = 128
HBM_FALLBACK_GBS = 6800.0
# Algorithmic bytes of the tree update of one iteration (PruneNodes over the
# pre-append tree, UpdateTree's rows, the V_U filter's candidate flags):
# per pre-append node 8 key + 4 region + 1 set + 1 inactivity count read, an
# 8-byte gather of its region's key and 1 set byte written; per appended row
# the state and control (4 n + 4 m), K 2, parent 4, key 8, region 4, set 1,
# inactivity count 1 and its region's key 8; one bit per candidate slot.
UPDATE_BYTES_PER_NODE = 23
UPDATE_PHASES = ("mark", "scan", "append", "prune")  # the append phase runs k_append, then k_stage


def update_row_bytes(n, m):
    return 4 * n + 4 * m + 28


# DRAM bytes (read + write) of the five update kernels of one iteration
# (k_mark, k_scan, k_append, k_stage, k_prune), from the ncu captures in
# profiles/ (each kernel from a cold L2, as ncu flushes caches between
# captured kernels): workload -> (iteration, bytes)
UPDATE_DRAM_BYTES = {
    "quad12_building1000": (100, 3745536),   # profiles/update_quad12_building1000.md
    "quad12_clutter1000": (300, 25009920),   # profiles/update_quad12_clutter1000.md
}


def hbm_peak():
    """(GB/s, basis): the copy bandwidth measured on this GPU pool
    (MEASURED_PEAKS.json beside this file), else the fallback figure."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "of measured (MEASURED_PEAKS.json hbm_gbs, STREAM-style copy)"
    except (OSError, ValueError, KeyError, TypeError):
        return HBM_FALLBACK_GBS, "of fallback (6.8 TB/s, one earlier GB300 measurement)"


def host_cpu():
    """Model, maximum clock and logical CPU count of the host."""
    model, mhz = None, None
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            k, _, v = line.partition(":")
            if k.strip() == "Model name" and not model:
                model = v.strip()
            elif k.strip() == "CPU max MHz":
                mhz = float(v.strip())
    except (OSError, ValueError, subprocess.SubprocessError):
        pass
    if mhz is None:
        try:
            with open("/sys/devices/system/cpu/cpu0/cpufreq/cpuinfo_max_freq") as f:
                mhz = int(f.read().strip()) / 1000.0
        except (OSError, ValueError):
            pass
    return {"model": model, "max_mhz": mhz, "logical_cpus": os.cpu_count()}


def fma_fields(achieved):
    """The device's FP32 FMA throughput measured now (kpx_fp32_fma_rate, one
    launch outside any timed region) and the achieved rate's fraction of it:
    the measured counterpart of the peak derived from unit counts and the
    clock."""
    import torch
    import paper_2602_02846_gb300 as kpx
    fma = kpx.fp32_fma_rate(2048, torch.cuda.current_stream())
    return {"peak_measured_fma": fma, "frac_of_measured_fma": achieved / fma if fma else None,
            "peak_measured_note": "FP32 FMA microbenchmark (kpx_fp32_fma_rate): 16 independent FMA "
                                  "chains per thread, 32 warps per SM"}

WORKLOADS = {
    "dubins6_forest300": dict(make=lambda seed: scenes.dubins_scene(seed),
                              desc="6D Dubins airplane, 300-column forest, RK4 h=0.02, 16^3x4 regions, "
                                   "cap 2^20, lambda 64"),
    "di6_boxes20": dict(make=lambda seed: scenes.di_scene(seed),
                        desc="6D double integrator, 20 boxes, Euler h=0.01, 8^3x2^3 regions, cap 32768, lambda 16"),
    "quad12_building1000": dict(make=lambda seed: scenes.quad_scene(seed),
                                desc="12D quadcopter, 1,000-box building, RK4 h=0.005, 16^3x4^3 regions, "
                                     "cap 2^22, lambda 128", ref_iters=3),
    # the same system and configuration among 1,000 boxes without the walls:
    # the tree grows past 2.5 M nodes in 400 iterations, where PruneNodes and
    # the append cover millions of nodes per iteration
    "quad12_clutter1000": dict(make=lambda seed: scenes.quad_scene(seed, clutter=1000, certify=False, walls=False,
                                                                   iterations=400),
                               desc="12D quadcopter, 1,000 boxes without walls, RK4 h=0.005, 16^3x4^3 regions, "
                                    "cap 2^22, lambda 128, 400 iterations", ref_iters=2),
}
BATCH_WORKLOADS = {
    "mixed_batch512": dict(count=512, desc="512 independent problems (DI / Dubins / quadcopter in turn), 10-1,000 "
                                           "boxes, tree caps 2^14-2^20, each family's grid and lambda, one "
                                           "launch per phase for all problems"),
}
SERVE_WORKLOADS = {
    "serve_poisson200": dict(rate=200.0, desc="request loop: Poisson arrivals at 200 queries/s drawn from the "
                                              "mixed-batch problem mix, admitted by device memory into per-class "
                                              "slots, iterations of all resident queries batched"),
    # the same loop under four times the load (context for where batching pays)
    "serve_poisson800": dict(rate=800.0, desc="request loop: Poisson arrivals at 800 queries/s drawn from the "
                                              "mixed-batch problem mix, admitted by device memory into per-class "
                                              "slots, iterations of all resident queries batched"),
}
REFINE_WORKLOADS = {
    "refine_quad4096": dict(count=4096, desc="adjoint refinement post-pass: 4,096 12D-quadcopter control sequences "
                                             "of 64-512 segments (10-60 RK4 steps each) among the 1,000-box "
                                             "building; one step = the objective and its gradient (forward with "
                                             "checkpoints every 32 steps + adjoint) for every sequence"),
}
# algorithmic FP32 work of the refinement objective and gradient (an FMA
# counts 2, a transcendental 1): per RK4 step and per box at each step
REFINE_OPS_RK4_STEP = 328.0        # 4 derivative evaluations (6 sin/cos + ~40 flops) + stage updates
REFINE_OPS_RK4_ADJOINT = 794.0     # 3 derivative + 4 vector-Jacobian evaluations + stage adjoints
REFINE_OPS_BOX_PENALTY = 22.0      # signed distance + softplus
REFINE_OPS_BOX_GRADIENT = 29.0     # signed distance + its gradient + sigmoid
REFINE_OPS_BOX_TEST = 13.0         # the squared outside distance and its comparison (every candidate box)
DEFAULT_WORKLOAD = "quad12_building1000"


def parse_args(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("kpx", "reference"), default="kpx")
    ap.add_argument("--workload", choices=sorted(WORKLOADS) + sorted(BATCH_WORKLOADS) + sorted(SERVE_WORKLOADS)
                    + sorted(REFINE_WORKLOADS), default=DEFAULT_WORKLOAD)
    ap.add_argument("--iters", type=int, default=0, help="planner iterations per step (0 = the config's)")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="budget of the oracle baseline sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="batch workloads: keep the default launch choices")
    ap.add_argument("--no-fused", action="store_true",
                    help="run every iteration as the phase kernels (KPX_FLAG_NO_FUSED; same results)")
    ap.add_argument("--no-slot-order", action="store_true",
                    help="propagate slots in index order, not sorted by step count (KPX_FLAG_NO_SLOT_ORDER; "
                         "same results)")
    ap.add_argument("--ttfs-seeds", type=int, default=8, help="problems (scene seeds) for time-to-first-solution")
    ap.add_argument("--ttfs-variant-seeds", type=int, default=100,
                    help="problems (scene seeds) per solvable variant for time-to-first-solution (default bench)")
    ap.add_argument("--serve-seconds", type=float, default=2.0, help="length of the served request stream")
    ap.add_argument("--serve-memory-gb", type=float, default=32.0, help="device arena of the request loop")
    ap.add_argument("--serve-slots", type=int, default=64, help="request-loop slots per dynamics class")
    ap.add_argument("--serve-round", type=int, default=4, help="iterations per request-loop round")
    ap.add_argument("--batch-count", type=int, default=0, help="problems of the batch workload (0 = its own)")
    ap.add_argument("--refine-count", type=int, default=0, help="trajectories of the refinement workload "
                                                                 "(0: the workload's 4,096)")
    return ap.parse_args(argv)


# ---------------------------------------------------------------------------
# distributed set-up (one process per GPU; replicas of independent problems)
# ---------------------------------------------------------------------------
def dist_setup(backend):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group(backend=backend)
    return world, rank, local


def allreduce(x, op, device):
    import torch
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized():
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op={"max": dist.ReduceOp.MAX, "sum": dist.ReduceOp.SUM}[op])
    return float(t.item())


def barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.barrier()


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.proc = None
        self.path = None
        self.gpu = gpu_index
        exe = shutil.which("nvidia-smi")
        if exe is None:
            return
        fd, self.path = tempfile.mkstemp(prefix="kpx_clocks_", suffix=".csv")
        os.close(fd)
        self.proc = subprocess.Popen([exe, "-i", str(gpu_index), "--query-gpu=" + self.FIELDS,
                                      "--format=csv,noheader,nounits", "-lms", "200"],
                                     stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "", 1).isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "", 1).isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for name, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "samples": len(rows), "reasons": sorted(reasons)}


# ---------------------------------------------------------------------------
# CPU baseline: the FP64 oracle on the same problem, bounded in time
# ---------------------------------------------------------------------------
def oracle_sample(prob, iters, budget_s):
    import oracle
    oracle.build()
    pl = oracle.Planner(prob)
    t0 = time.perf_counter()
    done = 0
    while done < iters:
        pl.iterate(1)
        done += 1
        if time.perf_counter() - t0 >= budget_s:
            break
    dt = time.perf_counter() - t0
    st = pl.state()
    return dict(valid=int(st["total_valid"]), candidates=int(st["total_candidates"]), iters=done, seconds=dt)


def refine_oracle_sample(batch, budget_s):
    """The FP64 oracle's objective + gradient on whole trajectories of the
    refinement batch, in order, until the budget is spent."""
    import oracle
    oracle.build()
    from paper_2602_02846_gb300 import refine
    prob = batch["problem"]
    spec = refine.default_cost(prob)
    t0 = time.perf_counter()
    done = steps = 0
    while done < batch["u"].shape[0]:
        n = int(batch["n_seg"][done])
        oracle.refine_grad(prob, spec, batch["x0"][done].astype(np.float64), batch["u"][done, :n].astype(np.float64),
                           batch["steps"][done, :n], obstacles=batch["obstacles"].astype(np.float64))
        steps += int(batch["steps"][done, :n].sum())
        done += 1
        if time.perf_counter() - t0 >= budget_s:
            break
    return dict(trajectories=done, steps=steps, seconds=time.perf_counter() - t0)


def run_reference(args):
    world, rank, local = dist_setup("gloo")
    if rank != 0:
        return 0
    if args.workload in REFINE_WORKLOADS:
        return run_refine_reference(args)
    if args.workload not in WORKLOADS:
        print(json.dumps({"impl": "reference", "unavailable": "the oracle arm times the single-problem and "
                          "refinement workloads; %s has no oracle leg" % args.workload}))
        return 0
    spec = WORKLOADS[args.workload]
    prob = spec["make"](args.seed)
    iters = args.iters or prob.iterations
    # a bounded sample: the oracle's first iterations of the same problem
    # (the quadcopter's first 3 take about 4 s on one core)
    per_step_iters = min(iters, spec.get("ref_iters", 40))
    for _ in range(args.warmup):
        oracle_sample(prob, min(per_step_iters, 2), 1e9)
    vals, secs = 0, 0.0
    for _ in range(args.steps):
        r = oracle_sample(prob, per_step_iters, 1e9)
        vals += r["valid"]
        secs += r["seconds"]
    value = vals / secs if secs > 0 else 0.0
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / max(1, args.steps),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "desc": spec["desc"], "iterations_per_step": per_step_iters,
                   "gpu_arm_iterations_per_step": iters, "same_iterations": per_step_iters == iters,
                   "note": "each step times the oracle's first %d of the %d iterations the GPU arm runs on the same "
                           "deterministic problem; both arms report valid expansions per second" % (per_step_iters,
                                                                                                   iters),
                   "seed": args.seed},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": "first %d iterations of the workload per step, single-threaded FP64 C oracle"
                                   % per_step_iters, "host": host_cpu()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
TTFS_VARIANTS = {
    "di6_16grid": dict(make=lambda seed: scenes.di_scene(seed, grid_pos=16),
                       desc="6D double integrator, 20 boxes, 16^3 x 2^3 regions, cap 32768, lambda 16"),
    "dubins6_forest30": dict(make=lambda seed: scenes.dubins_scene(seed, n_obstacles=30),
                             desc="6D Dubins airplane, 30-column forest, cap 2^20, lambda 64"),
    "quad12_room120": dict(make=lambda seed: scenes.quad_scene(seed, clutter=120, certify=False, walls=False,
                                                               tree_cap=1 << 16, lam=32),
                           desc="12D quadcopter, 120 boxes without walls, cap 2^16, lambda 32"),
}


def ttfs_block(kpx, make, seeds, iters, dev, stream):
    """Per problem: planned for `iters` iterations in one call (TTFS = device
    clock from the first iteration to the one that appended the first goal
    node), then reset and planned for the iterations that fit in 100 ms at
    its own measured rate (cost at 100 ms)."""
    times, costs100, solved = [], [], 0
    for sd in seeds:
        pk = kpx.Planner(make(sd), device=dev, stream=stream)
        s_k = pk.iterate(iters, stats=True)
        if s_k["first_solution_iter"] >= 0:
            solved += 1
            times.append(s_k["first_solution_ns"] / 1e6)
        t_iter_ms = max(1e-3, s_k["elapsed_ns"] / 1e6 / max(1, s_k["iter"]))
        pk.reset()
        s100 = pk.iterate(max(1, int(100.0 / t_iter_ms)), stats=True)
        if not math.isinf(s100["best_cost"]):
            costs100.append(float(s100["best_cost"]))
        pk.close()
    return {"problems": len(seeds), "solved": solved, "iterations": iters,
            "p50_ms": float(np.percentile(times, 50)) if times else None,
            "p99_ms": float(np.percentile(times, 99)) if times else None,
            "cost_at_100ms_median": float(np.median(costs100)) if costs100 else None,
            "solved_by_100ms": len(costs100),
            "note": "device clock from the first iteration to the iteration that appended the first goal node"}


def run_kpx(args):
    import torch
    world, rank, local = dist_setup("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import paper_2602_02846_gb300 as kpx
    kpx.load()
    spec = WORKLOADS[args.workload]
    prob = spec["make"](args.seed + rank)
    iters = args.iters or prob.iterations
    stream = torch.cuda.current_stream(dev)
    flags = (kpx.KPX_FLAG_NO_FUSED if args.no_fused else 0) | (kpx.KPX_FLAG_NO_SLOT_ORDER if args.no_slot_order
                                                                else 0)
    pl = kpx.Planner(prob, device=dev, stream=stream, flags=flags)

    # one step to learn the (deterministic) work of a step
    pl.reset()
    st = pl.iterate(iters, stats=True)
    valid_per_step = int(st["total_valid"])
    steps_per_step = int(st["total_steps"])
    tests_per_step = int(st["total_box_tests"])
    cand_per_step = int(st["total_candidates"])
    iters_done = int(st["iter"])
    for _ in range(max(0, args.warmup - 1)):
        pl.reset()
        pl.iterate(iters)
    torch.cuda.synchronize(dev)

    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > L2 (129 MB)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = ClockSampler(local)
    barrier()
    torch.cuda.synchronize(dev)
    for k in range(args.steps):
        flush.zero_()
        ev[k][0].record(stream)
        pl.reset()
        pl.iterate(iters)
        ev[k][1].record(stream)
    torch.cuda.synchronize(dev)
    barrier()
    clk = clocks.stop()
    ms = sum(a.elapsed_time(b) for a, b in ev)
    st2 = pl.iterate(0, stats=True)
    assert int(st2["total_valid"]) == valid_per_step, "steps are not identical"

    ms_max = allreduce(ms, "max", dev)
    valid_all = allreduce(valid_per_step * args.steps, "sum", dev)
    value = valid_all / (ms_max / 1e3)

    # launches of one step (kpx_graph_info): one graph launch per kpx_iterate
    # call, holding 1 fused launch plus 8 kernel launches per iteration the
    # fused kernel left to the loop (begin, propagate, stage, mark, scan, append,
    # prune, end); 8 per iteration without the fused kernel
    max_g, fused = pl.graph_info()
    plan = kpx.Planner.launch_plan(iters, max_g) if max_g else [1] * iters
    pl.reset()
    for g in plan:
        pl.iterate(g)
    fused_iters = int(pl.header().fused_iterations)
    graph_launches = len(plan) if max_g else 0
    if fused:
        launches_per_step = 1 + len(plan) + 8 * (iters - fused_iters)  # k_init (reset) first
    else:
        launches_per_step = 1 + 8 * iters

    # per-phase device time over one step (same launches, CUDA events on the
    # planner's stream; nothing synchronises inside the pass, so the host
    # stays ahead of the device and the events time the kernels alone)
    phase_ms = [0.0] * 7
    pl.reset()
    flush.zero_()
    evs = []
    for _ in range(iters):
        for ph in range(7):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            pl.debug_step(ph)
            b.record(stream)
            evs.append((ph, a, b))
    torch.cuda.synchronize(dev)
    for ph, a, b in evs:
        phase_ms[ph] += a.elapsed_time(b)
    # the same iterations again, untimed, reading each one's tree size,
    # winners kept and slots (the update's algorithmic bytes)
    upd_bytes, upd_bytes_at = 0, {}
    row = update_row_bytes(prob.n, prob.m)
    pl.reset()
    for it in range(iters):
        for ph in range(7):
            pl.debug_step(ph)
        h = pl.header()
        n_old = int(h.n_nodes) - int(h.n_kept)
        b_it = UPDATE_BYTES_PER_NODE * n_old + row * int(h.n_kept) + (int(h.n_slots) + 7) // 8
        upd_bytes += b_it
        upd_bytes_at[it] = b_it
    upd_ms = sum(phase_ms[kpx.PHASES.index(n)] for n in UPDATE_PHASES)
    hbm, hbm_basis = hbm_peak()
    upd_gbs = upd_bytes / (upd_ms / 1e3) / 1e9 if upd_ms > 0 else 0.0
    l2 = int(getattr(torch.cuda.get_device_properties(dev), "L2_cache_size", 0) or 0)
    work_set = UPDATE_BYTES_PER_NODE * int(st["n_nodes"]) + 8 * int(prob.n_regions)
    roofline_update = {
        "bound": "hbm",
        "kernel": "tree update: k_mark + k_scan + k_append + k_stage + k_prune (phase kernels, one after another)",
        "achieved": upd_gbs, "peak": hbm, "unit": "GB/s", "frac": upd_gbs / hbm if hbm else 0.0,
        "peak_basis": hbm_basis,
        "traffic": UPDATE_DRAM_BYTES[args.workload][1] if args.workload in UPDATE_DRAM_BYTES else None,
        "traffic_iteration": UPDATE_DRAM_BYTES[args.workload][0] if args.workload in UPDATE_DRAM_BYTES else None,
        "algorithmic_bytes_at_traffic_iteration": (upd_bytes_at.get(UPDATE_DRAM_BYTES[args.workload][0])
                                                   if args.workload in UPDATE_DRAM_BYTES else None),
        "traffic_note": "DRAM bytes of the five update kernels of one iteration (ncu capture, each kernel from a "
                        "cold L2; profiles/), beside the algorithmic bytes of the same iteration",
        "algorithmic_bytes_per_step": upd_bytes, "update_ms_per_step": upd_ms,
        "bytes_basis": "per iteration: %d B per pre-append node + %d B per appended row + 1 bit per candidate slot"
                      % (UPDATE_BYTES_PER_NODE, row),
        "working_set_bytes_end": work_set, "l2_bytes": l2,
        "l2_resident": bool(l2 and work_set < l2),
        "note": ("the update's working set (tree arrays and region keys) stays in L2 within a step, so this is an "
                 "L2/latency-bound figure reported against HBM bandwidth" if l2 and work_set < l2 else
                 "the tree outgrows L2: the update streams from HBM"),
    }
    prop_ms = phase_ms[1]
    prop_launch_ms = prop_ms / max(1, iters_done)
    ops_step = OPS_PER_STEP[prob.dyn] * steps_per_step + OPS_PER_BOX_TEST * tests_per_step
    sms = torch.cuda.get_device_properties(dev).multi_processor_count or SM_COUNT_FALLBACK
    peak_mhz = 2070.0
    peak = sms * FP32_LANES_PER_SM * 2 * peak_mhz * 1e6 / 1e12  # TFLOP/s
    achieved = (ops_step / max(1, iters_done)) / (prop_launch_ms / 1e3) / 1e12 if prop_ms > 0 else 0.0
    kernel, launch_ms = "k_propagate", prop_launch_ms
    traffic = PROPAGATE_DRAM_BYTES.get(args.workload)
    bound_note = "k_propagate is bound by instruction issue (FP32, SFU and compare work of the rollouts)"
    if fused and fused_iters == iters_done and graph_launches:
        # every iteration ran in the fused kernel: it is the step (the reset
        # kernel aside), so its time per launch comes from the timed region
        kernel, launch_ms = "k_fused (whole iterations, one cluster)", ms / args.steps / graph_launches
        achieved = ops_step / (ms / args.steps / 1e3) / 1e12
        traffic = FUSED_DRAM_BYTES.get(args.workload)
        bound_note = ("k_fused runs each iteration on one thread-block cluster: its time is the iteration's "
                      "dependent chain (the longest rollout, then the phases' cluster barriers), so the ALU "
                      "fraction below measures occupancy of the chip, not the kernel's distance from its bound")

    # end to end through the C ABI with host buffers
    e2e = None
    if not args.no_e2e:
        ws = pl.workspace
        pl.close()
        h2d = int(np.asarray(prob.obstacles).shape[0]) * 32 + 4 * prob.n
        d2h = 0
        barrier()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            p2 = kpx.Planner(prob, device=dev, stream=stream, workspace=ws, flags=flags)
            p2.iterate(iters)
            tr = p2.best_trajectory()
            hdr = ctypes.sizeof(kpx.kpx_device_header)
            d2h = hdr + ((len(tr["steps"]) + 1) * (prob.n + prob.m + 1) * 4 if tr is not None else 0)
            p2.close()
        torch.cuda.synchronize(dev)
        barrier()
        wall = time.perf_counter() - t0
        wall_max = allreduce(wall, "max", dev)
        e2e = {"value": valid_all / wall_max, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}
    else:
        pl.close()

    # time to first solution and cost at 100 ms over independent problems
    # (scene seeds) of this workload and of solvable variants of the three
    # systems (the literal Dubins forest and building do not solve)
    ttfs = ttfs_variants = None
    if args.ttfs_seeds > 0:
        seeds = [args.seed + 1000 * (rank + 1) + k for k in range(args.ttfs_seeds)]
        ttfs = ttfs_block(kpx, spec["make"], seeds, iters, dev, stream)
        if args.workload == DEFAULT_WORKLOAD and args.ttfs_variant_seeds > 0:
            vseeds = [args.seed + 1000 * (rank + 1) + 500 + k for k in range(args.ttfs_variant_seeds)]
            ttfs_variants = {name: dict(ttfs_block(kpx, v["make"], vseeds, 200, dev, stream), desc=v["desc"])
                             for name, v in TTFS_VARIANTS.items()}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        r = oracle_sample(prob, iters, args.cpu_seconds)
        cpu = {"value": r["valid"] / r["seconds"], "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": "first %d of %d iterations of the same problem (%d valid rollouts, %.1f s), "
                         "single-threaded FP64 C oracle" % (r["iters"], iters, r["valid"], r["seconds"]),
               "host": host_cpu()}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": args.workload, "desc": spec["desc"], "iterations_per_step": iters,
                       "iterations_run": iters_done, "seed": args.seed, "l2": "flushed between steps (256 MB write)",
                       "parallelism": "replicas (one independent problem per GPU)" if world > 1 else "single GPU",
                       "valid_per_step": valid_per_step, "candidates_per_step": cand_per_step,
                       "integration_steps_per_step": steps_per_step, "box_tests_per_step": tests_per_step,
                       "tree_nodes": int(st["n_nodes"]), "solution_cost": (None if math.isinf(st["best_cost"])
                                                                          else float(st["best_cost"]))},
            "roofline": {"bound": "alu", "bound_note": bound_note, "kernel": kernel, "achieved": achieved,
                         "peak": peak,
                         "unit": "TFLOP/s", "frac": achieved / peak if peak else 0.0,
                         "traffic": traffic,
                         "traffic_note": "DRAM bytes per launch of this kernel (ncu capture, profiles/); the "
                                         "kernel is ALU/latency-bound and its working set stays in L2",
                         "peak_basis": "%d SMs x %d FP32 lanes x 2 x %.0f MHz (max SM clock)"
                                       % (sms, FP32_LANES_PER_SM, peak_mhz),
                         **fma_fields(achieved),
                         "launch_ms": launch_ms,
                         "phase_kernels": {"propagate_launch_ms": prop_launch_ms,
                                           "propagate_achieved_tflops": (ops_step / max(1, iters_done))
                                           / (prop_launch_ms / 1e3) / 1e12 if prop_ms > 0 else 0.0,
                                           "phase_share": {n: round(t / sum(phase_ms), 4)
                                                           for n, t in zip(kpx.PHASES, phase_ms)},
                                           "note": "phase-by-phase pass over one step (kpx_debug_step)"}},
            "roofline_update": roofline_update,
            "launch_path": {"fused": bool(fused), "fused_iterations": fused_iters, "graph_launches": graph_launches,
                            "max_iterations_per_graph": max_g, "slot_order": not args.no_slot_order},
            "cpu_baseline": cpu,
            "e2e": e2e,
            "clocks": clk,
            "ttfs": ttfs,
            "ttfs_solvable_variants": ttfs_variants,
            "gpu_launches": launches_per_step * args.steps,
        }
        print(json.dumps(line))
    return 0


def run_batch(args):
    """Batched planning: one step = kpx_batch_reset + kpx_batch_iterate(I) over
    all problems; compared with the plain planner run problem by problem."""
    import torch
    world, rank, local = dist_setup("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import paper_2602_02846_gb300 as kpx
    kpx.load()
    spec = dict(BATCH_WORKLOADS[args.workload])
    if args.batch_count > 0:  # a smaller batch of the same mix (profiling)
        spec["count"] = args.batch_count
    iters = args.iters or 100
    probs = scenes.mixed_batch(spec["count"], seed=args.seed + 1000 * rank, iterations=iters)
    stream = torch.cuda.Stream(dev)
    with torch.cuda.stream(stream):
        batch = kpx.BatchPlanner(probs, device=dev, stream=stream)
    B = len(probs)

    def totals():
        v = steps = tests = 0
        ops = 0.0
        for i, pr in enumerate(probs):
            st = batch.member(i).iterate(0, stats=True)
            v += int(st["total_valid"])
            ops += OPS_PER_STEP[pr.dyn] * int(st["total_steps"]) + OPS_PER_BOX_TEST * int(st["total_box_tests"])
        return v, ops

    batch.reset()
    batch.iterate(iters)
    valid_per_step, ops_per_step = totals()
    # launch choices per dynamics class, timed on this state (results unchanged)
    tuned = None
    if not args.no_autotune:
        t0 = time.perf_counter()
        rep = batch.autotune(iters=4, blocks=(0, 2), scales=(0.5, 1.0, 2.0))
        names = {scenes.DI6: "di6", scenes.DUBINS6: "dubins6", scenes.QUAD12: "quad12"}
        tuned = {"%s/%s" % (names[c[0]], "rk4" if c[1] else "euler"):
                 {"propagate_blocks_per_sm": v["blocks"], "grid_scale": v["scale"], "ms_4_iterations": v["ms"]}
                 for c, v in rep.items()}
        tuned["seconds"] = time.perf_counter() - t0
    for _ in range(max(0, args.warmup - 1)):
        batch.reset()
        batch.iterate(iters)
    stream.synchronize()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = ClockSampler(local)
    barrier()
    torch.cuda.synchronize(dev)
    for k in range(args.steps):
        with torch.cuda.stream(stream):
            flush.zero_()
        ev[k][0].record(stream)
        batch.reset()
        batch.iterate(iters)
        ev[k][1].record(stream)
    torch.cuda.synchronize(dev)
    barrier()
    clk = clocks.stop()
    ms = sum(a.elapsed_time(b) for a, b in ev)
    assert totals()[0] == valid_per_step, "steps are not identical"
    # time to first solution of every problem in the last step (device clock
    # from the batch's first iteration)
    first = []
    for i in range(B):
        st = batch.member(i).iterate(0, stats=True)
        if st["first_solution_iter"] >= 0:
            first.append(st["first_solution_ns"] / 1e6)
    ms_max = allreduce(ms, "max", dev)
    valid_all = allreduce(valid_per_step * args.steps, "sum", dev)
    value = valid_all / (ms_max / 1e3)
    # the plain planner, problem by problem, on the same problems (same results)
    plain_ms = None
    if not args.no_e2e:
        singles = [kpx.Planner(pr, device=dev, stream=stream) for pr in probs]
        for pl in singles:
            pl.reset()
            pl.iterate(iters)
        stream.synchronize()
        with torch.cuda.stream(stream):
            flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for pl in singles:
            pl.reset()
            pl.iterate(iters)
        b.record(stream)
        torch.cuda.synchronize(dev)
        plain_ms = a.elapsed_time(b)
        for pl in singles:
            pl.close()
        del singles
    # end to end: create from host arrays, iterate, every best trajectory to host
    e2e = None
    if not args.no_e2e:
        ws = batch.workspace
        batch.close()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        h2d = d2h = 0
        for _ in range(args.steps):
            with torch.cuda.stream(stream):
                b2 = kpx.BatchPlanner(probs, device=dev, stream=stream)
            b2.iterate(iters)
            d2h = 0
            for i in range(B):
                tr = b2.member(i).best_trajectory()
                d2h += ctypes.sizeof(kpx.kpx_device_header)
                if tr is not None:
                    d2h += (len(tr["steps"]) + 1) * (probs[i].n + probs[i].m + 1) * 4
            b2.close()
        torch.cuda.synchronize(dev)
        wall = time.perf_counter() - t0
        h2d = sum(int(np.asarray(pr.obstacles).shape[0]) * 32 for pr in probs)
        e2e = {"value": valid_all / allreduce(wall, "max", dev), "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h}
    else:
        batch.close()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count or SM_COUNT_FALLBACK
    peak = sms * FP32_LANES_PER_SM * 2 * 2070.0 * 1e6 / 1e12
    achieved = ops_per_step / (ms / args.steps / 1e3) / 1e12
    if rank == 0:
        kinds = {}
        for pr in probs:
            kinds[pr.name] = kinds.get(pr.name, 0) + 1
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": args.workload, "desc": spec["desc"], "problems": B, "families": kinds,
                       "iterations_per_step": iters, "seed": args.seed, "l2": "flushed between steps (256 MB write)",
                       "valid_per_step": valid_per_step},
            "plain_sequential": None if plain_ms is None else {
                "value": valid_per_step / (plain_ms / 1e3), "ms_per_step": plain_ms,
                "note": "the same problems planned one after another with kpx_create/kpx_iterate (identical "
                        "results, so equal solution cost)"},
            "batch_speedup_vs_plain": None if plain_ms is None else plain_ms / (ms / args.steps),
            "autotuned": tuned,
            "roofline": {"bound": "alu", "kernel": "k_b_propagate (whole iteration time: a lower bound)",
                         "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                         "traffic": None, **fma_fields(achieved)},
            "ttfs": {"problems": B, "solved": len(first),
                     "p50_ms": float(np.percentile(first, 50)) if first else None,
                     "p99_ms": float(np.percentile(first, 99)) if first else None,
                     "note": "device clock from the batch's first iteration"},
            "cpu_baseline": None, "e2e": e2e, "clocks": clk,
            # per step: one reset kernel per problem, then per iteration begin, snapshot, mark, scan,
            # prefix, prune, end and one propagate + one append per dynamics class
            "gpu_launches": args.steps * (B + iters * (7 + 2 * len({(pr.dyn, pr.integ) for pr in probs}))),
        }
        print(json.dumps(line))
    return 0


def run_serve(args):
    """The request loop (continuous batching) on one stream of Poisson
    arrivals; a step serves the whole stream in real time.  Beside it, the
    same stream through the plain planner one query at a time."""
    import torch
    world, rank, local = dist_setup("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import paper_2602_02846_gb300 as kpx
    from paper_2602_02846_gb300 import serve
    kpx.load()
    spec = SERVE_WORKLOADS[args.workload]
    budget = args.iters or 64
    stream_reqs = scenes.poisson_requests(spec["rate"], args.serve_seconds, seed=args.seed + 1000 * rank)
    sizes = [kpx.kpx_workspace_size(p) for _, p in stream_reqs]

    def requests():
        return [serve.Request(i, p, t, budget, nbytes=n) for i, ((t, p), n) in enumerate(zip(stream_reqs, sizes))]

    stream = torch.cuda.Stream(dev)
    srv = serve.Server.create(int(args.serve_memory_gb * (1 << 30)), slots_per_class=args.serve_slots, device=dev,
                              stream=stream, iters_per_round=args.serve_round)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    warm = requests()[:min(len(stream_reqs), 48)]
    for _ in range(args.warmup):
        srv.serve(warm, realtime=False)
    clocks = ClockSampler(local)
    walls, results = [], None
    srv.rounds = srv.resident_sum = srv.admits = srv.trajectories = 0
    barrier()
    for k in range(args.steps):
        with torch.cuda.stream(stream):
            flush.zero_()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        results = srv.serve(requests(), realtime=True)
        torch.cuda.synchronize(dev)
        walls.append(time.perf_counter() - t0)
    barrier()
    clk = clocks.stop()
    wall = sum(walls)
    summ = serve.summarize(results, srv.offset, walls[-1])
    valid_step = sum(o.total_valid for o in results)
    value = allreduce(valid_step * args.steps, "sum", dev) / allreduce(wall, "max", dev)
    rounds, resident = srv.rounds, srv.resident_sum
    launches = (rounds * (args.serve_round * (7 + 2 * 3) + 1) + srv.admits * 5 + srv.trajectories * 2)
    srv.batch.close()
    plain = None
    if not args.no_e2e:
        t0 = time.perf_counter()
        pouts = serve.serve_plain(requests(), device=dev, stream=stream, iters_per_round=args.serve_round)
        pwall = time.perf_counter() - t0
        plain = serve.summarize(pouts, 0.0, pwall)
        plain["wall_s"] = pwall
        same = sum(1 for a, b in zip(results, pouts) if a.cost == b.cost and a.iterations == b.iterations)
        plain["identical_costs"] = same
    if rank == 0:
        h2d = sum(int(np.asarray(p.obstacles).size) * 4 + int(np.asarray(p.start).size) * 4 for _, p in stream_reqs)
        d2h = sum(0 if o.trajectory is None else
                  (len(o.trajectory["steps"]) + 1) * (o.trajectory["states"].shape[1] + 1) * 4 for o in results)
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * wall / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": args.workload, "desc": spec["desc"], "rate_qps": spec["rate"],
                       "stream_seconds": args.serve_seconds, "requests": len(stream_reqs),
                       "iterations_per_request": budget, "iterations_per_round": args.serve_round,
                       "slots_per_class": args.serve_slots, "arena_gb": args.serve_memory_gb, "seed": args.seed,
                       "l2": "flushed before each served stream (256 MB write)",
                       "timing": "host wall clock of serve() over the whole stream (arrivals in real time)"},
            "serving": summ,
            "mean_resident": resident / rounds if rounds else None,
            "plain_one_at_a_time": plain,
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "note": "the request loop is end to end: problems from host arrays, trajectories to host"},
            "cpu_baseline": None, "clocks": clk, "gpu_launches": launches,
        }
        print(json.dumps(line))
    return 0


def run_refine_reference(args):
    spec = dict(REFINE_WORKLOADS[args.workload])
    if args.refine_count:
        spec["count"] = args.refine_count
    batch = scenes.refine_batch(spec["count"], seed=args.seed)
    budget = max(1.0, args.cpu_seconds / max(1, args.steps))
    refine_oracle_sample(batch, 0.1)
    trajs = steps = 0
    secs = 0.0
    for _ in range(args.steps):
        r = refine_oracle_sample(batch, budget)
        trajs += r["trajectories"]
        steps += r["steps"]
        secs += r["seconds"]
    value = trajs / secs if secs > 0 else 0.0
    unit = "trajectory gradients/s"
    line = {
        "impl": "reference", "metric": "trajectory gradients/s", "value": value, "unit": unit, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / max(1, args.steps),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "desc": spec["desc"], "seed": args.seed},
        "cpu_baseline": {"value": value, "unit": unit, "cores": 1, "kind": "oracle",
                         "sample": "%d whole trajectories (%d RK4 steps) of the batch, FP64 objective + reverse-mode "
                                   "gradient, single-threaded C" % (trajs, steps)},
        "e2e": {"value": value, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def run_refine(args):
    """Objective + adjoint gradient of 4,096 control sequences per step."""
    import torch
    world, rank, local = dist_setup("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import paper_2602_02846_gb300 as kpx
    from paper_2602_02846_gb300 import refine
    kpx.load()
    spec = dict(REFINE_WORKLOADS[args.workload])
    if args.refine_count:
        spec["count"] = args.refine_count
    data = scenes.refine_batch(spec["count"], seed=args.seed + 1000 * rank)
    prob = data["problem"]
    batch = refine.Batch(prob, data["x0"], data["u"], data["steps"], data["n_seg"], obstacles=data["obstacles"],
                         device=dev)
    cost = refine.default_cost(prob)
    stream = torch.cuda.current_stream(dev)
    n_steps = int(data["steps"].sum())
    M = int(data["obstacles"].shape[0])
    for _ in range(args.warmup):
        refine.evaluate(batch, cost, grad=True)
    torch.cuda.synchronize(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = ClockSampler(local)
    barrier()
    torch.cuda.synchronize(dev)
    for k in range(args.steps):
        flush.zero_()
        ev[k][0].record(stream)
        J, g = refine.evaluate(batch, cost, grad=True)
        ev[k][1].record(stream)
    torch.cuda.synchronize(dev)
    barrier()
    clk = clocks.stop()
    ms = sum(a.elapsed_time(b) for a, b in ev)
    finite = bool(torch.isfinite(J).all().item() and torch.isfinite(g).all().item())
    ms_max = allreduce(ms, "max", dev)
    value = allreduce(spec["count"] * args.steps, "sum", dev) / (ms_max / 1e3)
    # the forward and the backward kernels timed apart (same launches)
    a, b, c = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    flush.zero_()
    a.record(stream)
    refine.evaluate(batch, cost)
    b.record(stream)
    refine.evaluate(batch, cost, grad=True)
    c.record(stream)
    torch.cuda.synchronize(dev)
    fwd_ms, both_ms = a.elapsed_time(b), b.elapsed_time(c)
    # the arithmetic executed in one step: the RK4 steps (forward,
    # recomputation, adjoint) and the box tests the kernels counted (the last
    # evaluate above: candidates from the box grid, terms within the far
    # distance)
    f_cand, f_near, b_cand, b_near = refine.box_tests(batch)
    ops = (n_steps * (2 * REFINE_OPS_RK4_STEP + REFINE_OPS_RK4_ADJOINT)
           + (f_cand + b_cand) * REFINE_OPS_BOX_TEST
           + f_near * (REFINE_OPS_BOX_PENALTY - REFINE_OPS_BOX_TEST + 1.0)
           + b_near * (REFINE_OPS_BOX_GRADIENT - REFINE_OPS_BOX_TEST + 1.0))
    # the objective as it defines the work: every box's term at every step
    ops_objective = n_steps * (2 * REFINE_OPS_RK4_STEP + REFINE_OPS_RK4_ADJOINT
                               + M * (REFINE_OPS_BOX_PENALTY + REFINE_OPS_BOX_GRADIENT))
    sms = torch.cuda.get_device_properties(dev).multi_processor_count or SM_COUNT_FALLBACK
    peak = sms * FP32_LANES_PER_SM * 2 * 2070.0 * 1e6 / 1e12
    achieved = ops / (ms / args.steps / 1e3) / 1e12
    objective_rate = ops_objective / (ms / args.steps / 1e3) / 1e12
    # end to end: controls, start states and step counts from pinned host
    # memory, objective and gradient back to the host
    e2e = None
    if not args.no_e2e:
        hu = torch.from_numpy(data["u"]).pin_memory()
        hx = torch.from_numpy(data["x0"]).pin_memory()
        hs = torch.from_numpy(data["steps"]).pin_memory()
        hJ = torch.empty(spec["count"], dtype=torch.float32).pin_memory()
        hg = torch.empty_like(hu).pin_memory()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            batch.u.copy_(hu, non_blocking=True)
            batch.x0.copy_(hx, non_blocking=True)
            batch.steps.copy_(hs, non_blocking=True)
            J, g = refine.evaluate(batch, cost, grad=True)
            hJ.copy_(J, non_blocking=True)
            hg.copy_(g, non_blocking=True)
        torch.cuda.synchronize(dev)
        wall = time.perf_counter() - t0
        e2e = {"value": allreduce(spec["count"] * args.steps, "sum", dev) / allreduce(wall, "max", dev),
               "unit": "trajectory gradients/s",
               "h2d_bytes_per_step": int(hu.numel() * 4 + hx.numel() * 4 + hs.numel() * 4),
               "d2h_bytes_per_step": int(hJ.numel() * 4 + hg.numel() * 4)}
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        r = refine_oracle_sample(data, args.cpu_seconds)
        cpu = {"value": r["trajectories"] / r["seconds"], "unit": "trajectory gradients/s", "cores": 1,
               "kind": "oracle", "sample": "the first %d trajectories (%d RK4 steps) of the batch, FP64 objective "
                                           "+ reverse-mode gradient, single-threaded C (%.1f s)"
                                           % (r["trajectories"], r["steps"], r["seconds"])}
    if rank == 0:
        line = {
            "metric": "trajectory gradients/s", "value": value, "unit": "trajectory gradients/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": args.workload, "desc": spec["desc"], "trajectories": spec["count"],
                       "rk4_steps_per_step": n_steps, "boxes": M, "seed": args.seed,
                       "l2": "flushed between steps (256 MB write)", "all_finite": finite},
            "roofline": {"bound": "alu", "kernel": "k_refine_forward<true> + k_refine_backward (one step)",
                         "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                         "traffic": None,
                         "ops_note": "executed arithmetic: per RK4 step forward %.0f + recomputation %.0f + adjoint "
                                     "%.0f; %.0f per candidate box (the box grid's, counted by the kernels), plus "
                                     "%.0f (penalty) or %.0f (gradient) per box within the far distance"
                                     % (REFINE_OPS_RK4_STEP, REFINE_OPS_RK4_STEP, REFINE_OPS_RK4_ADJOINT,
                                        REFINE_OPS_BOX_TEST, REFINE_OPS_BOX_PENALTY - REFINE_OPS_BOX_TEST + 1.0,
                                        REFINE_OPS_BOX_GRADIENT - REFINE_OPS_BOX_TEST + 1.0),
                         "box_tests_per_step": {"objective_candidates": f_cand, "objective_terms": f_near,
                                                "gradient_candidates": b_cand, "gradient_terms": b_near,
                                                "every_box": n_steps * M},
                         "objective_rate_tflops": objective_rate,
                         "objective_rate_note": "every box's term at every step, %.0f + %.0f operations each, over "
                                                "the same time: the rate of the objective as defined"
                                                % (REFINE_OPS_BOX_PENALTY, REFINE_OPS_BOX_GRADIENT),
                         "peak_basis": "%d SMs x %d FP32 lanes x 2 x 2070 MHz (max SM clock)"
                                       % (sms, FP32_LANES_PER_SM),
                         **fma_fields(achieved),
                         "forward_only_ms": fwd_ms, "forward_and_backward_ms": both_ms},
            "cpu_baseline": cpu, "e2e": e2e, "clocks": clk,
            "gpu_launches": 2 * args.steps,
        }
        print(json.dumps(line))
    return 0


def main(argv=None):
    args = parse_args(argv)
    if args.impl == "reference":
        return run_reference(args)
    if args.workload in BATCH_WORKLOADS:
        return run_batch(args)
    if args.workload in SERVE_WORKLOADS:
        return run_serve(args)
    if args.workload in REFINE_WORKLOADS:
        return run_refine(args)
    return run_kpx(args)


if __name__ == "__main__":
    sys.exit(main())
