#!/usr/bin/env python
"""Throughput of the DI-LBM hot path on one GB300 (MLUPS, HBM roofline).

One step = one time step of the whole hot path on the lattice: the fused
pull-stream + DI-collide sweep over every node (with the solid fraction and
the per-tile force partials), the per-particle FP64 force/torque reduction
with Wan-Turek repulsion, and the rigid-body update with re-binning.

Default workload: 4096 x 4096 periodic box with 2048 free discs (radius
uniform in [6, 12], rho_s/rho_f = 1.2, g = 1e-6, tau = 0.8, interface width 2),
FP32 deviation storage.  The populations (1.2 GB for A and B) are far larger
than L2, so no flush is needed between steps.

Prints one JSON line.  ``--impl reference`` times the FP64 CPU oracle instead
(host cores, a down-scaled copy of the same workload per step).
Multi-GPU (torchrun): every rank advances its own lattice (independent
problems, no data-path collective); the value is the node updates of all
ranks over the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "MLUPS"
BYTES_PER_NODE = {"fp32": 72, "fp16": 36, "bf16": 36}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=4000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="dilbm", choices=["dilbm", "reference"])
    ap.add_argument("--workload", default="periodic", choices=["periodic", "sedimentation", "cylinder", "batch", "serve"])
    ap.add_argument("--storage", default="fp32", choices=["fp32", "fp16", "bf16"])
    ap.add_argument("--method", default="di", choices=["di", "ps"],
                    help="coupling: the paper's DI-LBM, or its PS-LBM comparison (periodic/cylinder/sedimentation)")
    ap.add_argument("--size", type=int, default=4096, help="periodic box edge")
    ap.add_argument("--decompose", action="store_true",
                    help="periodic/settling workloads under torchrun: split one lattice into strips over the "
                         "ranks (strong scaling) instead of one replica per rank")
    ap.add_argument("--particles", type=int, default=2048)
    ap.add_argument("--e2e-steps", type=int, default=200)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-table", action="store_true",
                    help="time the oracle on 1 and all host cores for the cylinder, settling and suspension workloads")
    ap.add_argument("--requests", type=int, default=300, help="serve: leading requests of the stream")
    ap.add_argument("--max-jobs", type=int, default=64, help="serve: jobs resident at once")
    ap.add_argument("--jobs-log", default=None,
                    help="serve: write one JSON line per cylinder job (parameters, FP16 vs FP32 drag) to this file")
    ap.add_argument("--macro-steps", type=int, default=64, help="serve: steps per macro-step")
    ap.add_argument("--shape", default=None,
                    help="sweep launch shape warps,blocks_per_sm (default: the autotuner's)")
    return ap.parse_args()


def make_problem(args, rank=0):
    from paper_2106_08950_gb300 import workloads as W
    if args.workload == "periodic":
        p = W.periodic_suspension(n=args.size, count=args.particles, seed=3 + 1000 * rank)
        cfg = {"workload": f"periodic suspension {args.size}x{args.size}, {args.particles} discs r~U[6,12], "
                           f"rho_s/rho_f=1.2, g=1e-6, tau=0.8, eps=2"}
    elif args.workload == "sedimentation":
        p = W.sedimentation()
        cfg = {"workload": "settling disc 400x2000 closed box, r=12, rho_s/rho_f=1.5, g=1e-5, tau=0.8, eps=2"}
    else:
        p = W.cylinder_drag()
        cfg = {"workload": "cylinder drag 200x100, r=10, U=0.05, Re=20, eps=2"}
    if args.method == "ps":
        p.method = W.METHOD_PS
        cfg["method"] = "PS-LBM, SP collision (Eqs. 7-12), exact covered cell fraction"
    else:
        cfg["method"] = "DI-LBM (Eqs. 13-19)"
    return p, cfg


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while running."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        mhz, maxes, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                mhz.append(float(parts[0]))
                maxes.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(n)
        if not mhz:
            return None
        return {"sm_mhz": statistics.median(mhz), "sm_max_mhz": max(maxes), "reasons": sorted(reasons),
                "samples": len(mhz)}


# ---------------------------------------------------------------- dist
def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def init_dist(world, backend):
    if world > 1:
        import torch.distributed as dist
        if not dist.is_initialized():
            dist.init_process_group(backend=backend)
        return dist
    return None


def max_over_ranks(dist, value, device=None):
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(dist, value, device=None):
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def gather_lists(dist, items):
    """Every rank's list, concatenated in rank order (the list itself at N=1)."""
    if dist is None:
        return list(items)
    out = [None] * dist.get_world_size()
    dist.all_gather_object(out, list(items))
    return [v for part in out for v in part]


def shard(items, rank, world):
    """Rank ``rank``'s share of independent work items (every world-th)."""
    return list(items)[rank::world]


def barrier(dist):
    if dist is not None:
        dist.barrier()


# ---------------------------------------------------------------- oracle arms
def force_model_name(fm: int) -> str:
    return {0: "Eq. 18 as printed", 1: "momentum exchange"}.get(int(fm), str(fm))


def cpu_model() -> str:
    """The host CPU's model name (lscpu), for the oracle timings."""
    import subprocess
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    return "unknown"


def oracle_mlups(prob, seconds: float, max_steps: int = 1_000_000, min_steps: int = 2, threads: int = 0):
    """Time the FP64 oracle as it stands on the host cores (``threads``: 0 =
    all of them)."""
    from oracle import oracle as O
    full = O.max_threads() if threads else 0
    sim = O.OracleSim(prob, phi_cutoff=4 * prob.eps, threads=threads)
    try:
        sim.step(1)                      # warm-up: first-touch of the arrays
        t0 = time.perf_counter()
        n = 0
        while n < max_steps and (n < min_steps or time.perf_counter() - t0 < seconds):
            sim.step(1)
            n += 1
        dt = time.perf_counter() - t0
        cores = O.max_threads()
    finally:
        sim.close()
        if full:
            O.set_threads(full)
    return prob.nx * prob.ny * n / dt / 1e6, n, dt, cores


def cpu_table(args):
    """The oracle on the host cores, single-threaded and on every core, for
    the cylinder workload in full (2000 steps), the settling disc (2000
    steps) and the periodic suspension (20 steps); each measurement is capped
    at --cpu-seconds x 10 of wall time and reports the steps it ran."""
    from oracle import oracle as O
    from paper_2106_08950_gb300 import workloads as W
    cases = [("cylinder 200x100, r=10, Re=20", W.cylinder_drag(), 2000),
             ("settling disc 400x2000, r=12", W.sedimentation(), 2000),
             ("periodic suspension 4096x4096, 2048 discs", W.periodic_suspension(), 20)]
    allc = O.max_threads()
    rows = []
    for name, prob, steps in cases:
        for threads in (1, allc):
            v, n, dt, cores = oracle_mlups(prob, args.cpu_seconds * 10, max_steps=steps, min_steps=1,
                                           threads=threads)
            rows.append({"workload": name, "threads": cores, "steps_run": n, "steps_asked": steps,
                         "seconds": dt, "MLUPS": v})
            print(json.dumps(rows[-1]), flush=True)
    print(json.dumps({"cpu_table": rows, "cpu_model": cpu_model(), "cores": allc}), flush=True)
    return 0


def reference_arm(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    from paper_2106_08950_gb300 import workloads as W
    prob, cfg = make_problem(args)
    # each step: one oracle step of a 512^2 copy of the workload (same
    # radius, density and area-fraction distributions)
    n_small = 512
    count = max(1, round(len(prob.particles) * (n_small / max(prob.nx, 1)) ** 2)) if args.workload == "periodic" else 0
    small = (W.periodic_suspension(n=n_small, count=count, seed=3) if args.workload == "periodic" else prob)
    small.method = prob.method
    from oracle import oracle as O
    sim = O.OracleSim(small, phi_cutoff=4 * small.eps)
    for _ in range(args.warmup):
        sim.step(1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        sim.step(1)
    dt = time.perf_counter() - t0
    v = small.nx * small.ny * args.steps / dt / 1e6
    sample = (f"{small.nx}x{small.ny} copy with {len(small.particles)} discs per step"
              if small is not prob else "the full workload per step")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "MLUPS", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": cfg,
            "cpu_baseline": {"value": v, "unit": "MLUPS", "cores": O.max_threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": v, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- GPU arm
def measured_peak_hbm():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def measured_traffic(key):
    """DRAM bytes per sweep launch from a committed ncu summary, if it was
    taken on the current kernel source (else None)."""
    import glob
    import hashlib
    import re
    src = os.path.join(ROOT, "paper_2106_08950_gb300", "csrc", "dilbm_kernels.cuh")
    with open(src, "rb") as fh:
        sha = hashlib.sha256(fh.read()).hexdigest()[:16]
    for path in glob.glob(os.path.join(ROOT, "profiles", "*.md")):
        with open(path) as fh:
            for m in re.finditer(r"<!-- traffic (\S+) (\d+) sha256=(\w+) -->", fh.read()):
                if m.group(1) == key and m.group(3) == sha:
                    return int(m.group(2))
    return None


def strips_arm(args):
    """One lattice split into horizontal strips over the ranks (strong
    scaling): each rank sweeps its rows and the ranks exchange the rows beside
    each cut and the per-particle force sums every step (NCCL)."""
    import torch
    from paper_2106_08950_gb300 import strips as S

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = init_dist(world, "nccl")
    dev = torch.device("cuda", local)
    prob, cfg = make_problem(args, 0)               # the same lattice on every rank
    stream = torch.cuda.Stream(device=dev)
    sim = S.DecomposedSimulation(prob, storage=args.storage, stream=stream)
    sim.step(args.warmup)
    sim.sync()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    barrier(dist)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    l0 = sim.sim.launches
    with torch.cuda.stream(stream):
        ev0.record(stream)
        sim.step(args.steps)
        ev1.record(stream)
    sim.sync()
    torch.cuda.synchronize()
    barrier(dist)
    clk = clocks.stop()
    ms = max_over_ranks(dist, ev0.elapsed_time(ev1), dev)
    launches = int(sum_over_ranks(dist, sim.sim.launches - l0, dev))
    value = prob.nx * prob.ny * args.steps / (ms / 1e3) / 1e6
    line = {"metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "strong", "vs_baseline": None,
            "dtype": {"fp32": "f32", "fp16": "f16-storage/f32-math", "bf16": "bf16-storage/f32-math"}[args.storage],
            "data": "synthetic",
            "config": dict(cfg, storage=args.storage, nodes=prob.nx * prob.ny, particles=len(prob.particles),
                           force_model=force_model_name(prob.force_model),
                           strips=[list(S.strip_rows(prob.ny, world, r)) for r in range(world)],
                           l2="populations exceed L2; no flush", parallelism=f"strips x{world} (NCCL halo rows + "
                                                                          "per-particle force all-reduce)"),
            "roofline": None, "gpu_launches": launches, "e2e": None, "clocks": clk}
    if rank == 0:
        print(json.dumps(line), flush=True)
    sim.close()
    dist.destroy_process_group()
    return 0


def gpu_arm(args):
    import ctypes as C

    import torch
    from paper_2106_08950_gb300 import dilbm as D
    from paper_2106_08950_gb300 import workloads as W

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = init_dist(world, "nccl")
    dev = torch.device("cuda", local)
    prob, cfg = make_problem(args, rank)
    stream = torch.cuda.Stream(device=dev)
    sim = D.Simulation(prob, storage=args.storage, stream=int(stream.cuda_stream))
    nodes = prob.nx * prob.ny

    # warm-up, then the launch shape the autotuner picks for this lattice
    sim.step(args.warmup)
    sim.sync()
    if args.shape:
        shape = tuple(int(v) for v in args.shape.split(","))
        sim.set_shape(*shape)
    else:
        shape = sim.autotune()
    sim.step(2)
    sim.sync()

    # ---- device-resident throughput: steps replayed from CUDA graphs,
    # bracketed by CUDA events on the launching stream
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    barrier(dist)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    l0 = sim.launches
    with torch.cuda.stream(stream):
        ev0.record(stream)
        sim.step(args.steps)
        ev1.record(stream)
    sim.sync()
    torch.cuda.synchronize()
    barrier(dist)
    launches = sim.launches - l0
    ms = ev0.elapsed_time(ev1)
    # ---- the sweep kernel alone: events around each launch (direct launches)
    sim.set_timing(True)
    sim.step(min(args.steps, 400))
    sweep_ms, sweep_n = sim.sweep_time()
    sim.set_timing(False)
    clk = clocks.stop()
    ms_max = max_over_ranks(dist, ms, dev)
    value = nodes * args.steps * world / (ms_max / 1e3) / 1e6

    # ---- end to end through the C ABI with host buffers: each step uploads
    # the particle state from pinned host memory, advances one step and reads
    # the forces and state back (a host-coupled particle loop).
    npart = len(prob.particles)
    e2e = None
    if npart > 0 and args.e2e_steps > 0:
        import numpy as np
        F = np.zeros((npart, 3))
        host_state = torch.empty(npart * C.sizeof(D.Particle), dtype=torch.uint8).pin_memory()
        arr = (D.Particle * npart).from_address(host_state.data_ptr())
        F_pinned = torch.zeros(npart * 3, dtype=torch.float64).pin_memory()
        Fp = np.frombuffer((C.c_double * (npart * 3)).from_address(F_pinned.data_ptr()), dtype=np.float64)
        sim.L.dilbm_forces(sim.h, Fp.ctypes.data, None, C.cast(arr, C.c_void_p))
        barrier(dist)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            D.check(sim.L.dilbm_set_particles(sim.h, arr, npart))
            D.check(sim.L.dilbm_step(sim.h, 1))
            D.check(sim.L.dilbm_forces(sim.h, Fp.ctypes.data, None, C.cast(arr, C.c_void_p)))
        dt = time.perf_counter() - t0
        dt = max_over_ranks(dist, dt, dev)
        h2d = npart * (8 * 8 + 4)
        d2h = npart * 3 * 8 + npart * (8 * 8 + 4) + 4
        e2e = {"value": nodes * args.e2e_steps * world / dt / 1e6, "unit": "MLUPS",
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
               "loop": "per step: dilbm_set_particles(host) + dilbm_step(1) + dilbm_forces(host)"}

    # ---- roofline of the dominant kernel (the lattice sweep)
    peak, peak_kind = measured_peak_hbm()
    per_launch_ms = sweep_ms / max(sweep_n, 1)
    alg_bytes = BYTES_PER_NODE[args.storage] * nodes
    achieved = alg_bytes / (per_launch_ms / 1e3) / 1e9
    traffic = measured_traffic(f"{args.workload}:{args.storage}:{prob.nx}x{prob.ny}" + (":ps" if prob.method == W.METHOD_PS else ""))
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": traffic, "peak_kind": peak_kind,
            "kernel": "sweep_kernel", "sweep_ms_per_launch": per_launch_ms,
            "sweep_share_of_step": per_launch_ms / (ms / args.steps) if ms > 0 else None,
            "algorithmic_bytes_per_launch": alg_bytes}

    line = {"metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp32": "f32", "fp16": "f16-storage/f32-math", "bf16": "bf16-storage/f32-math"}[args.storage],
            "data": "synthetic",
            "config": dict(cfg, storage=args.storage, nodes=nodes, particles=npart,
                           force_model=force_model_name(prob.force_model),
                           launch_shape={"warps_per_block": shape[0], "blocks_per_sm": shape[1],
                                         "by": "--shape" if args.shape else "autotuner"},
                           l2="populations 9x2 planes exceed L2; no flush",
                           parallelism=f"replicas x{world}" if world > 1 else "single GPU"),
            "roofline": roof, "gpu_launches": int(sum_over_ranks(dist, launches, dev)), "e2e": e2e, "clocks": clk}

    # ---- the oracle on the host cores, rank 0 at N=1 only
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, n, dt, cores = oracle_mlups(prob, args.cpu_seconds)
        v1, n1, dt1, _ = oracle_mlups(prob, args.cpu_seconds, threads=1, min_steps=1)
        line["cpu_baseline"] = {"value": v, "unit": "MLUPS", "cores": cores, "kind": "oracle",
                                "sample": f"{n} steps of the full workload ({dt:.1f} s), " + (
                                    "cell fractions within r + 0.71" if prob.method == W.METHOD_PS
                                    else "phi cutoff 4 widths"),
                                "single_thread": {"value": v1, "unit": "MLUPS", "cores": 1,
                                                  "sample": f"{n1} steps of the full workload ({dt1:.1f} s)"},
                                "cpu_model": cpu_model()}
    if rank == 0:
        print(json.dumps(line), flush=True)
    sim.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


def batch_arm(args):
    """64 uneven lattices (seed 4) advanced together by the batched launch,
    against the same lattices stepped one at a time."""
    import torch
    from paper_2106_08950_gb300 import dilbm as D
    from paper_2106_08950_gb300 import workloads as W

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = init_dist(world, "nccl")
    dev = torch.device("cuda", local)
    jobs = W.batch_lattices(seed=4 + 1000 * rank)
    nodes = sum(j.nodes for j in jobs)
    stream = torch.cuda.Stream(device=dev)
    sh = int(stream.cuda_stream)
    members = [D.Simulation(j, storage=args.storage, stream=sh) for j in jobs]
    batch = D.Batch(members)
    batch.step(args.warmup)
    batch.sync()
    if args.shape:
        shape = tuple(int(v) for v in args.shape.split(","))
        batch.set_shape(*shape)
    else:
        shape = batch.autotune()
    batch.step(2)
    batch.sync()

    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    barrier(dist)
    torch.cuda.synchronize()
    l0 = batch.launches
    t0 = time.perf_counter()
    batch.step(args.steps)
    batch.sync()
    dt = time.perf_counter() - t0
    launches = batch.launches - l0
    clk = clocks.stop()
    dt = max_over_ranks(dist, dt, dev)
    total_nodes = sum_over_ranks(dist, nodes, dev)        # each rank has its own lattices
    value = total_nodes * args.steps / dt / 1e6

    # the batched sweep alone, timed by CUDA events (direct launches)
    k_t = max(10, min(args.steps, 200))
    batch.set_timing(True)
    batch.step(k_t)
    sweep_ms, sweep_n = batch.sweep_time()
    batch.set_timing(False)
    batch.sync()

    # the same lattices one at a time, each for the same number of steps
    k_alone = max(10, min(args.steps, 200))
    alone = [D.Simulation(j, storage=args.storage, stream=sh) for j in jobs]
    for a in alone:
        a.step(args.warmup)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for a in alone:
        a.step(k_alone)
    for a in alone:
        a.sync()
    dt_alone = time.perf_counter() - t0
    dt_alone = max_over_ranks(dist, dt_alone, dev)
    alone_value = total_nodes * k_alone / dt_alone / 1e6

    peak, peak_kind = measured_peak_hbm()
    per_launch = sweep_ms / max(sweep_n, 1)
    alg = BYTES_PER_NODE[args.storage] * nodes
    achieved = alg / (per_launch / 1e3) / 1e9
    line = {"metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp32": "f32", "fp16": "f16-storage/f32-math", "bf16": "bf16-storage/f32-math"}[args.storage],
            "data": "synthetic",
            "config": {"workload": "batch of 64 uneven lattices (seed 4): nx log-U[128,1024], ny log-U[128,2048], "
                                   "cylinder or sedimentation jobs, 1-32 discs r U[5,15], Re log-U[10,100]",
                       "storage": args.storage, "nodes": nodes, "nodes_all_ranks": total_nodes, "lattices": len(jobs),
                       "force_model": ", ".join(sorted({force_model_name(j.force_model) for j in jobs})),
                       "particles": sum(len(j.particles) for j in jobs),
                       "launch": "one batched sweep + one batched particle launch per step, CUDA-graph replay",
                       "launch_shape": {"warps_per_block": shape[0], "blocks_per_sm": shape[1],
                                        "by": "--shape" if args.shape else "autotuner"},
                       "l2": f"{nodes * BYTES_PER_NODE[args.storage] / 1e6:.0f} MB of populations per step"},
            "one_at_a_time": {"value": alone_value, "unit": "MLUPS", "steps": k_alone,
                              "speedup_of_batch": value / alone_value},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "traffic": measured_traffic(f"batch:{args.storage}:{len(jobs)}x{nodes}"),
                         "peak_kind": peak_kind, "kernel": "sweep_kernel (batched)",
                         "sweep_ms_per_launch": per_launch, "algorithmic_bytes_per_launch": alg},
            "gpu_launches": int(sum_over_ranks(dist, launches, dev)), "e2e": None, "clocks": clk}
    if rank == 0:
        print(json.dumps(line), flush=True)
    for a in alone:
        a.close()
    batch.close()
    for m in members:
        m.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


def percentile(xs, q):
    import numpy as np
    return float(np.percentile(np.asarray(xs, dtype=float), q)) if len(xs) else None


def replay_served(reqs, storage, args, D):
    """Replay the arrival schedule in real time into a server; returns the
    per-request latencies, results and the server's counters."""
    srv = D.Server(storage, max_jobs=args.max_jobs, macro_steps=args.macro_steps)
    t_base = srv.clock()
    nxt = 0
    ids = {}
    while True:
        now = srv.clock() - t_base
        while nxt < len(reqs) and reqs[nxt].arrival_s <= now:
            r = reqs[nxt]
            ids[srv.submit(r.problem, r.steps, arrival=t_base + r.arrival_s, mean_window=r.steps // 4)] = nxt
            nxt += 1
        st = srv.progress()
        if st.running == 0 and st.queued == 0:
            if nxt == len(reqs):
                break
            time.sleep(max(0.0, reqs[nxt].arrival_s - (srv.clock() - t_base)))
    lat, res, first, last = {}, {}, None, 0.0
    stored = {}
    for jid, k in ids.items():
        js = srv.status(jid)
        if js.state != D.JOB_DONE:
            raise RuntimeError(f"request {k} ended in state {js.state} (error {js.error})")
        lat[k] = js.finished - js.arrival
        last = max(last, js.finished - t_base)
        stored[k] = js.storage
        res[k] = srv.result(jid, with_mean=True)
    first = reqs[0].arrival_s
    srv_stats = st
    srv.close()
    return lat, res, last - first, srv_stats, stored


def replay_single(reqs, storage, D, stream):
    """The plain single-instance path: one Simulation at a time in arrival
    order (dilbm_create, dilbm_step(n), dilbm_forces), in real time."""
    t_base = time.perf_counter()
    lat, res, launches = {}, {}, 0
    for k, r in enumerate(reqs):
        now = time.perf_counter() - t_base
        if now < r.arrival_s:
            time.sleep(r.arrival_s - now)
        sim = D.Simulation(r.problem, storage=storage, stream=stream)
        sim.step(r.steps)
        F, _, S = sim.forces()
        launches += sim.launches
        sim.close()
        lat[k] = time.perf_counter() - t_base - r.arrival_s
        res[k] = (F, None, S)
    return lat, res, time.perf_counter() - t_base - reqs[0].arrival_s, launches


def job_rows(reqs, res_a, res_b):
    """Per cylinder job: its parameters and the FP16 (res_a) vs FP32 (res_b)
    mean drag of its worst disc, for diagnosing the reduced-precision error."""
    rows = []
    for k, r in enumerate(reqs):
        p = r.problem
        if not p.particles or not p.particles[0].fixed:
            continue
        Fa, Fb = res_a[k][1], res_b[k][1]
        u = abs(p.west.ux)
        m = int(abs(Fa[:, 0] - Fb[:, 0]).argmax())
        d = 2.0 * max(q.r for q in p.particles)
        rows.append({"request": k, "name": p.name, "nx": p.nx, "ny": p.ny, "discs": len(p.particles),
                     "steps": r.steps, "tau": p.tau, "U": u, "Re": u * d / ((p.tau - 0.5) / 3.0),
                     "worst_disc": m, "r": p.particles[m].r, "x": p.particles[m].x,
                     "Fx_fp16": float(Fa[m, 0]), "Fx_fp32": float(Fb[m, 0]),
                     "max_abs_Fx_fp32": float(abs(Fb[:, 0]).max()),
                     "cd_err": float(abs(Fa[m, 0] - Fb[m, 0]) / (0.5 * u * u * 2.0 * p.particles[m].r))})
    return rows


def drag_errors(reqs, res_a, res_b):
    """Per cylinder job, on the mean F_x over its last quarter of steps: the
    largest difference over its discs in drag-coefficient units,
    |dF_x| / (rho U^2 D / 2) (Eq. 21 with the inlet speed U and the disc's
    diameter D), and the same relative to the largest |F_x| of the job."""
    cd, rel = [], []
    for k, r in enumerate(reqs):
        p = r.problem
        if not p.particles or not p.particles[0].fixed:
            continue
        Fa, Fb = res_a[k][1], res_b[k][1]
        u = abs(p.west.ux)
        dcd = [abs(Fa[m, 0] - Fb[m, 0]) / (0.5 * u * u * 2.0 * q.r) for m, q in enumerate(p.particles)]
        cd.append(float(max(dcd)))
        scale = abs(Fb[:, 0]).max()
        if scale > 0:
            rel.append(float(abs(Fa[:, 0] - Fb[:, 0]).max() / scale))
    return cd, rel


def serve_arm(args):
    """The Poisson request stream (seed 5, 50 requests/s) served by continuous
    batching in FP16 and FP32 deviation storage, against the plain
    single-instance FP32 path on the same arrivals."""
    import torch
    from paper_2106_08950_gb300 import dilbm as D
    from paper_2106_08950_gb300 import workloads as W

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = init_dist(world, "nccl")
    dev = torch.device("cuda", local)
    # replicas: rank k serves every world-th request of the stream
    reqs = shard(W.request_stream(count=args.requests * world), rank, world)
    work = sum(r.problem.nx * r.problem.ny * r.steps for r in reqs)
    total_work = sum_over_ranks(dist, work, dev)        # node updates of all ranks' requests
    stream = torch.cuda.Stream(device=dev)
    sh = int(stream.cuda_stream)
    # warm-up: one small job through each path (module load, graph capture)
    warm = [W.Request(0.0, 10, W.cylinder_drag())]
    replay_served(warm, "fp16", args, D)
    replay_single(warm, "fp32", D, sh)

    arms = {}
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    barrier(dist)
    for name, storage in (("served_auto", "auto"), ("served_fp16", "fp16"), ("served_fp32", "fp32")):
        lat, res, span, st, stored = replay_served(reqs, storage, args, D)
        span = max_over_ranks(dist, span, dev)
        arms[name] = {"lat": lat, "res": res, "span": span, "launches": st.launches, "stored": stored,
                      "host": {"macro_steps": st.macro_steps, "busy_s": st.busy_seconds, "form_s": st.form_seconds,
                               "admit_s": st.admit_seconds, "wait_s": st.wait_seconds,
                               "retire_s": st.retire_seconds}}
        barrier(dist)
    lat, res, span, launches = replay_single(reqs, "fp32", D, sh)
    span = max_over_ranks(dist, span, dev)
    arms["single_fp32"] = {"lat": lat, "res": res, "span": span, "launches": launches}
    clk = clocks.stop()

    def summary(a):
        lv = gather_lists(dist, a["lat"].values())          # every rank's requests
        out = {"value": total_work / a["span"] / 1e6, "unit": "MLUPS", "p50_s": percentile(lv, 50),
               "p99_s": percentile(lv, 99), "makespan_s": a["span"],
               "gpu_launches": int(sum_over_ranks(dist, a["launches"], dev))}
        if "host" in a:
            out["server_time"] = a["host"]
        return out

    sa, s16, s32, s1 = (summary(arms["served_auto"]), summary(arms["served_fp16"]), summary(arms["served_fp32"]),
                        summary(arms["single_fp32"]))
    d16, r16 = drag_errors(reqs, arms["served_fp16"]["res"], arms["served_fp32"]["res"])
    if args.jobs_log:
        with open(f"{args.jobs_log}.rank{rank}" if world > 1 else args.jobs_log, "w") as fh:
            for row in job_rows(reqs, arms["served_fp16"]["res"], arms["served_fp32"]["res"]):
                row["auto_storage"] = int(arms["served_auto"]["stored"][row["request"]])
                fh.write(json.dumps(row) + "\n")
    d16, r16 = gather_lists(dist, d16), gather_lists(dist, r16)
    da, ra = drag_errors(reqs, arms["served_auto"]["res"], arms["served_fp32"]["res"])
    da, ra = gather_lists(dist, da), gather_lists(dist, ra)
    n16 = sum_over_ranks(dist, sum(1 for v in arms["served_auto"]["stored"].values() if v == D.FP16_DEV), dev)
    ncyl = sum_over_ranks(dist, sum(1 for k, r in enumerate(reqs) if r.problem.particles and r.problem.particles[0].fixed
                                    and arms["served_auto"]["stored"][k] == D.FP16_DEV), dev)
    parts_in = sum(len(r.problem.particles) for r in reqs)
    import numpy as np
    same = all(np.array_equal(arms["served_fp32"]["res"][k][0], arms["single_fp32"]["res"][k][0]) and
               np.array_equal(arms["served_fp32"]["res"][k][2], arms["single_fp32"]["res"][k][2])
               for k in range(len(reqs)))
    same = sum_over_ranks(dist, 0.0 if same else 1.0, dev) == 0.0
    def drag_summary(d, r):
        return {"jobs": len(d), "quantity": "mean F_x over each cylinder job's last quarter of steps, vs served FP32",
                "cd_units": {"median": percentile(d, 50), "p90": percentile(d, 90), "max": max(d) if d else None,
                             "frac_le_1e-3": sum(1 for v in d if v <= 1e-3) / max(1, len(d))},
                "relative": {"median": percentile(r, 50), "p90": percentile(r, 90), "max": max(r) if r else None,
                             "frac_le_1e-3": sum(1 for v in r if v <= 1e-3) / max(1, len(r))}}

    line = {"metric": METRIC, "value": sa["value"], "unit": "MLUPS", "n_gpus": world, "steps": len(reqs),
            "warmup": 1, "ms_per_step": None, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f16/f32-storage (per job)/f32-math", "data": "synthetic",
            "config": {"workload": f"served: the first {len(reqs) * world} requests of a Poisson stream "
                                   "(seed 5, 50 requests/s): cylinder or sedimentation jobs, nx, ny log-U[128,2048], "
                                   "1-64 discs r U[5,15], steps log-U[1k,20k]; replayed in real time",
                       "storage": "auto: FP16 deviations where tau <= 0.6 and the discs cover <= 5% of the "
                                  "lattice, else FP32",
                       "jobs_in_fp16": int(n16), "cylinder_jobs_in_fp16": int(ncyl),
                       "node_updates": total_work, "max_jobs": args.max_jobs,
                       "force_model": ", ".join(sorted({force_model_name(r.problem.force_model) for r in reqs})),
                       "macro_steps": args.macro_steps, "admission": "FIFO by job slots and free device memory",
                       "l2": "resident lattices exceed L2 once a few large jobs run; no flush",
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
            "latency": {"p50_s": sa["p50_s"], "p99_s": sa["p99_s"]},
            "server_time": sa.get("server_time"),
            "served_fp16_all_jobs": s16, "served_fp32": s32, "single_instance_fp32": s1,
            "gain_over_single_fp32": {"mlups": sa["value"] / s1["value"], "p50": s1["p50_s"] / sa["p50_s"],
                                      "p99": s1["p99_s"] / sa["p99_s"]},
            "drag_error_auto_vs_fp32": drag_summary(da, ra),
            "drag_error_fp16_all_jobs_vs_fp32": drag_summary(d16, r16),
            "fp32_served_equals_single_bitwise": same,
            "roofline": None, "gpu_launches": sa["gpu_launches"],
            "e2e": {"value": sa["value"], "unit": "MLUPS", "h2d_bytes_per_step": None, "d2h_bytes_per_step": None,
                    "h2d_bytes_per_request": parts_in * 72 // max(1, len(reqs)),
                    "d2h_bytes_per_request": parts_in * (72 + 24) // max(1, len(reqs)),
                    "note": "the served value is end to end: host job descriptions in, host results out"},
            "clocks": clk}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return reference_arm(args)
    if args.cpu_table:
        return cpu_table(args)
    if args.workload == "batch":
        return batch_arm(args)
    if args.workload == "serve":
        return serve_arm(args)
    if args.decompose and dist_env()[0] > 1:
        return strips_arm(args)
    return gpu_arm(args)


if __name__ == "__main__":
    sys.exit(main())
