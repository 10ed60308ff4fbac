#!/usr/bin/env python
"""Throughput of the HJ level-set solve (Algorithm 1 of arXiv 2204.05520) on GB300.

One benchmark step = one complete solve of the workload (all time steps of
the tau schedule) with the value arrays resident in HBM.  The default workload
is the 4D Dubins car BRT on an 80x80x40x64 grid (16.4M nodes), ENO2 + TVD-RK2,
CFL 0.8, t in [0, 3] (265 time steps).  The metric is grid-point updates per
second (nodes x time steps / device time), reported with the fraction of the
measured HBM copy bandwidth reached by the fused stage kernel.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
  python bench.py --impl reference ...   # the FP64 CPU oracle on the host cores

Under torchrun every rank solves its own copy of the workload (independent
solves, weak scaling); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import dataclasses
import hashlib
import glob
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

METRIC = "grid-point updates/s"
UNIT = "updates/s"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "dram_traffic.txt")
FALLBACK_HBM_GBS = 6800.0
NOMINAL_HBM_GBS = 7900.0   # GB300 HBM3e, nominal
# time-to-reach sweeping (Algorithm 2) on the grids of the paper's tables
TTR_WORKLOADS = tuple("ttr_%s_%d" % (m, n) for m in ("dubins3d", "dubinscar4d") for n in (60, 80, 100))


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--workload", choices=("dubinscar4d", "dubins3d", "rel6d", "dubinscar4d_reach_avoid",
                                           "batch512", "served") + TTR_WORKLOADS,
                    default="dubinscar4d")
    ap.add_argument("--rates", default="10,30,100,300,1000,2000",
                    help="served workload: Poisson arrival rates (req/s)")
    ap.add_argument("--window", type=float, default=3.0,
                    help="served workload: seconds of arrivals per rate (at most 2000 requests)")
    ap.add_argument("--budget-gb", type=float, default=150.0)
    ap.add_argument("--max-resident-mnodes", type=float, default=0.0,
                    help="served workload: cap on the grid nodes of resident solves, millions (0: none)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="headline workload only (skip the other configurations)")
    ap.add_argument("--dissipation", choices=("global", "local"), default="global",
                    help="Lax-Friedrichs dissipation: grid alpha or each node's own alpha")
    ap.add_argument("--stage-pass", choices=("auto", "plane", "bulk"), default="auto",
                    help="stage-pass kernel of the single solve (auto: the faster one for the model)")
    ap.add_argument("--host-loop", action="store_true",
                    help="step the time loop from the host (same kernels; for profilers)")
    return ap.parse_args()


def rank_info():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def hbm_peak():
    try:
        with open(PEAKS_FILE) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


# sources that define the stage pass and the model instantiations it is
# profiled on: a DRAM-traffic record holds only while these are unchanged
STAGE_SOURCES = ("odp_common.cuh", "hj_device.cuh", "hj_kernels.cuh", "hj_plane.cuh", "hj_bulk.cuh",
                 "kern_dubins.cu", "kern_rel6d.cu", "odp_api.cu")   # odp_api.cu: the launch geometry


def kernel_sources_sha() -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2204_05520_gb300", "csrc")
    for p in [os.path.join(csrc, f) for f in STAGE_SOURCES]:
        with open(p, "rb") as fh:
            h.update(os.path.basename(p).encode())
            h.update(fh.read())
    return h.hexdigest()[:16]


def dram_traffic(workload: str):
    """ncu DRAM bytes (read + write) per stage launch recorded for this
    workload in profiles/dram_traffic.txt ("<workload> <sources sha>
    <bytes>" lines), if the kernel sources are unchanged since the capture;
    else None."""
    try:
        sha = kernel_sources_sha()
        with open(TRAFFIC_FILE) as fh:
            for line in fh:
                f = line.split()
                if len(f) == 3 and f[0] == workload and f[1] == sha:
                    return float(f[2])
    except Exception:
        pass
    return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup(world: int, use_cuda: bool):
    if world <= 1:
        return None
    import torch.distributed as dist

    dist.init_process_group(backend="nccl" if use_cuda else "gloo")
    return dist


def max_over_ranks(dist, value: float, device) -> float:
    if dist is None:
        return value
    import torch

    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(dist):
    if dist is not None:
        dist.barrier()


# ---------------------------------------------------------------------------
# CPU oracle: baseline sample and the reference arm
# ---------------------------------------------------------------------------

def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo), or the machine type."""
    import platform

    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.split(":")[0].strip().lower() == "model name":
                return "%s (%s)" % (line.split(":", 1)[1].strip(), platform.machine())
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                key = line.split(":")[0].strip().lower()
                if key in ("model name", "cpu model", "hardware"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return platform.machine()


def oracle_sample(problem, n_steps: int):
    """Time the FP64 oracle on the full workload, stopped by its step limit
    after `n_steps` time steps; returns (updates/s, seconds, threads, steps)."""
    import oracle

    oracle.build()
    l = problem.target_values()
    t0 = time.perf_counter()
    r = oracle.solve(problem, l=l, max_steps=n_steps, raise_on_error=False)
    secs = time.perf_counter() - t0
    steps = int(r["steps"].sum())
    return problem.points * steps / secs, secs, oracle.num_threads(), steps


def oracle_ttr_sample(problem, n_sweeps: int):
    """Time the FP64 oracle's sweeps on the full grid, stopped by its sweep cap
    after `n_sweeps` sweeps; returns (updates/s, seconds, threads, sweeps)."""
    import oracle

    oracle.build()
    t0 = time.perf_counter()
    r = oracle.ttr(problem, max_sweeps=n_sweeps, raise_on_error=False)
    secs = time.perf_counter() - t0
    # the Gauss-Seidel sweep is sequential: one core
    return problem.points * r["sweeps"] / secs, secs, 1, r["sweeps"]


def run_reference_ttr(args, problem):
    for _ in range(args.warmup):
        oracle_ttr_sample(problem, 1)
    total_updates, total_s, threads = 0.0, 0.0, 1
    for _ in range(args.steps):
        ups, secs, threads, _ = oracle_ttr_sample(problem, 1)
        total_updates += ups * secs
        total_s += secs
    value = total_updates / total_s
    sample = "one sweep of the full %s grid (%d nodes) per benchmark step" % (problem.name, problem.points)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * total_s / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": problem.name, "method": "Lax-Friedrichs sweeping"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": sample, "cpu_model": cpu_model()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def oracle_solve_estimate(problem):
    """Seconds the FP64 oracle would take for the whole solve of ``problem``:
    the time of one step (the oracle stopped after 3 and after 1 steps, the
    difference halved, so that fixed per-call costs cancel) times the step
    count of its CFL schedule (the last step of each tau segment clipped)."""
    import math

    import oracle

    oracle.build()
    l = problem.target_values()
    secs = []
    for k in (1, 3):
        t0 = time.perf_counter()
        r = oracle.solve(problem, l=l, max_steps=k, raise_on_error=False)
        secs.append(time.perf_counter() - t0)
    per_step = max(secs[1] - secs[0], 0.0) / 2.0
    dz = [(problem.hi[d] - problem.lo[d]) / (problem.n[d] if problem.periodic[d] else problem.n[d] - 1)
          for d in range(problem.ndim)]
    dt = problem.cfl / sum(float(r["alpha"][d]) / dz[d] for d in range(problem.ndim))
    tau = problem.tau
    steps = sum(math.ceil((tau[k + 1] - tau[k]) / dt - 1e-9) for k in range(len(tau) - 1))
    return per_step * steps, steps, oracle.num_threads()


def run_reference_solves(args):
    """Reference arm of the batched and served workloads (solves/s): the
    oracle solves the workload's problems one at a time; each benchmark step
    takes the next problem, timing one full time step and extrapolating to
    its step count (a whole oracle solve of a large grid takes minutes)."""
    from paper_2204_05520_gb300 import inputs

    if args.workload == "batch512":
        problems = inputs.batch_problems(count=512, seed=0)
        metric, name = "batched solves/s", "batch512_dubins3d"
    else:
        problems = [p for _, p in inputs.served_requests(100.0, count=max(40, args.steps + args.warmup), seed=1)]
        metric, name = "served solves/s (saturation) with p50/p99 latency", "served_poisson_dubins3d_dubinscar4d"
    for i in range(args.warmup):
        oracle_solve_estimate(problems[i % len(problems)])
    total, threads = 0.0, 1
    for i in range(args.steps):
        est, _, threads = oracle_solve_estimate(problems[(args.warmup + i) % len(problems)])
        total += est
    value = args.steps / total
    sample = ("%d problems of the workload solved one at a time: the time of one full step of each (oracle "
              "stopped after 3 and after 1 steps), times its CFL step count" % args.steps)
    line = {
        "impl": "reference", "metric": metric, "value": value, "unit": "solves/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": name},
        "cpu_baseline": {"value": value, "unit": "solves/s", "cores": threads, "kind": "oracle",
                         "sample": sample, "cpu_model": cpu_model()},
        "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_reference(args):
    rank, world, _ = rank_info()
    if rank != 0:
        return 0
    from paper_2204_05520_gb300 import inputs

    if args.workload in ("batch512", "served"):
        return run_reference_solves(args)
    problem = inputs.workload(args.workload)
    if args.workload in TTR_WORKLOADS:
        return run_reference_ttr(args, problem)
    for _ in range(args.warmup):
        oracle_sample(problem, 1)
    total_updates, total_s, threads = 0.0, 0.0, 1
    for _ in range(args.steps):
        ups, secs, threads, steps = oracle_sample(problem, 1)
        total_updates += ups * secs
        total_s += secs
    value = total_updates / total_s
    sample = "one time step of the full %s grid (%d nodes) per benchmark step" % (
        problem.name, problem.points)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * total_s / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": problem.name},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": sample, "cpu_model": cpu_model()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

# FP32 lane operations per node of one stage of the ENO2 Lax-Friedrichs
# update (Algorithm 1), counted from the scheme: per axis 7 differences, 2
# magnitude comparisons and 2 selects (the ENO choice), 2 fused multiply-adds
# (p-, p+), 2 additions (their sum and difference) and 2 fused multiply-adds
# (drift or input-bound term, dissipation) = 17; plus the update (1 fused
# multiply-add; RK2 stage 2 adds the Heun average, 2, and the BRT min, 1).
ALU_OPS_PER_AXIS = {1: 8, 2: 17}   # upwind: 2 differences, 2 additions, 2 + 2 fused multiply-adds
GB300_FP32_LANE_OPS = 152 * 128 * 2.07e9   # SMs x FP32 lanes x maximum SM clock


def alu_ops_per_node_step(problem) -> float:
    per_stage = ALU_OPS_PER_AXIS[problem.space_order] * problem.ndim
    if problem.time_order == 2:
        return (per_stage + 1) + (per_stage + 1 + 2 + (1 if problem.set_kind == "brt" else 0))
    return per_stage + 1 + (1 if problem.set_kind == "brt" else 0)


def measure_solve(problem, steps, warmup, stream=None):
    """Device time of `steps` whole solves (one CUDA graph each) of `problem`
    with its values resident; returns a dict of figures."""
    import torch

    from paper_2204_05520_gb300 import odp

    stream = stream or torch.cuda.Stream()
    N = problem.points
    l_dev = torch.from_numpy(problem.target_values()).cuda()
    with odp.Grid.for_problem(problem, stream=stream) as grid:
        grid.set_target(l_dev)
        with torch.cuda.stream(stream):
            for _ in range(warmup):
                grid.solve_problem(problem)
        st = odp.solve_status(grid.handle)
        torch.cuda.synchronize()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(steps):
            grid.solve_problem(problem)
        ev1.record(stream)
        torch.cuda.synchronize()
        odp.solve_status(grid.handle)
        ms = ev0.elapsed_time(ev1) / steps
        stages = (1, 2) if problem.time_order == 2 else (0,)
        stage_ms = [odp.time_stage(grid.handle, k, reps=10) for k in stages]
    n_steps = int(st["steps"])
    return {"workload": problem.name, "nodes": N, "time_steps_per_solve": n_steps, "ms_per_solve": ms,
            "solves_per_s": 1000.0 / ms, "updates_per_s": N * n_steps / (ms / 1000.0),
            "alg_bytes_per_solve": float(st["bytes"]),
            "roofline_frac": float(st["bytes"]) / (ms / 1000.0) / 1e9 / hbm_peak()[0],
            "alu_frac": alu_ops_per_node_step(problem) * N * n_steps / (ms / 1000.0) / GB300_FP32_LANE_OPS,
            "stage_ms_isolated": stage_ms, "gpu_launches_per_solve": int(st["launches"])}


def extra_workloads(args):
    """The other configurations beside the headline, on one GPU: the 3D
    Dubins car (41x41x36), the 6D relative model (24^6), 512 batched
    Dubins3D solves and the served Poisson stream at three rates."""
    from paper_2204_05520_gb300 import inputs

    out = {}
    out["dubins3d_41x41x36"] = measure_solve(inputs.workload("dubins3d"), 50, 5)
    out["rel6d_24^6"] = measure_solve(inputs.workload("rel6d"), 2, 1)
    out["batch512_dubins3d"] = measure_batch(3, 2)
    points, single = measure_served([10.0, 30.0, 100.0], 2.0, args.budget_gb)
    out["served_poisson"] = {"rates": points, "window_s": 2.0, "budget_gb": args.budget_gb,
                             "saturation_solves_per_s": max((pt["solves_per_s"] or 0.0) for pt in points),
                             "one_at_a_time_solves_per_s": single}
    return out


def run_ours(args):
    import numpy as np
    import torch

    from paper_2204_05520_gb300 import _build, inputs, odp

    rank, world, local = rank_info()
    torch.cuda.set_device(local)
    dist = dist_setup(world, True)
    _build.build()
    odp.load()
    device = torch.device("cuda", local)
    problem = inputs.workload(args.workload)
    if args.dissipation == "local":
        problem = dataclasses.replace(problem, dissipation="local")
    N = problem.points
    l_host = problem.target_values()
    stream = torch.cuda.Stream()
    l_dev = torch.from_numpy(l_host).to(device)
    grid = odp.Grid.for_problem(problem, stream=stream)
    if args.host_loop:
        odp.set_loop_mode(grid.handle, True)
    odp.set_stage_pass(grid.handle, {"auto": 0, "plane": 1, "bulk": 2}[args.stage_pass])
    grid.set_target(l_dev)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            grid.solve_problem(problem)
    st = odp.solve_status(grid.handle)
    steps_per_solve = int(st["steps"])
    launches_per_solve = int(st["launches"])   # the once-per-solve launches included
    bytes_per_solve = float(st["bytes"])

    sampler = ClockSampler(local)
    torch.cuda.synchronize()
    barrier(dist)
    sampler.start()
    time.sleep(0.3)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        grid.solve_problem(problem)
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier(dist)
    clocks = sampler.stop()
    ms_total = ev0.elapsed_time(ev1)
    odp.solve_status(grid.handle)   # raises if the device flagged an error
    ms_total = max_over_ranks(dist, ms_total, device)
    ms_per_step = ms_total / args.steps
    value = world * N * steps_per_solve / (ms_per_step / 1000.0)

    # Roofline of the time loop, live over the timed region: the algorithmic
    # bytes of every stage pass divided by the event-timed region, so the
    # time of the small dt/alpha kernels (and the Rel6D heading-rate pass,
    # which stops reading once its ceiling is reached) counts against the
    # stage pass.  The stage pass alone (events around 20
    # back-to-back launches on the grid's stream) is reported beside it.
    stages = (1, 2) if problem.time_order == 2 else (0,)
    stage_ms = [odp.time_stage(grid.handle, s, reps=20) for s in stages]
    stage_launches = steps_per_solve * len(stages)
    peak, peak_kind = hbm_peak()
    achieved = bytes_per_solve / (ms_per_step / 1000.0) / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "frac_of_nominal": achieved / NOMINAL_HBM_GBS,
                "traffic": dram_traffic(problem.name),
                "kernel": "%s (whole time loop timed)" % (
                    "k_stage_bulk" if (args.stage_pass == "bulk" or (args.stage_pass == "auto" and
                                                                       problem.ndim >= 4))
                    else "k_stage_plane"), "peak_source": peak_kind,
                "alg_bytes_per_launch": bytes_per_solve / stage_launches,
                "avg_launch_ms": ms_per_step / stage_launches,
                "stage_ms_isolated": stage_ms}

    # end to end through the C ABI with host buffers (pinned), copies timed
    e2e = None
    if not args.no_e2e:
        l_pin = torch.from_numpy(l_host).pin_memory()
        out_pin = torch.empty_like(l_pin).pin_memory()
        grid.solve_problem(problem)
        grid.readback(out_pin)
        torch.cuda.synchronize()
        barrier(dist)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            grid.set_target(l_pin)
            grid.solve_problem(problem)
            grid.readback(out_pin)
        t_e2e = time.perf_counter() - t0
        t_e2e = max_over_ranks(dist, t_e2e, device)
        e2e = {"value": world * N * steps_per_solve * args.steps / t_e2e, "unit": UNIT,
               "h2d_bytes_per_step": 4 * N, "d2h_bytes_per_step": 4 * N,
               "ms_per_step": 1000.0 * t_e2e / args.steps}
        grid.set_target(l_dev)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        ups, secs, threads, nst = oracle_sample(problem, 5)
        cpu = {"value": ups, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": "%d time steps of the full %s grid (%d nodes), %.1f s" % (
                   nst, problem.name, N, secs),
               "cpu_model": cpu_model()}
        if args.workload in ("dubins3d", "dubinscar4d"):
            # the same oracle on one core (one time step of the full grid)
            import oracle

            oracle.set_threads(1)
            ups1, secs1, _, nst1 = oracle_sample(problem, 1 if N > 1e6 else 10)
            oracle.set_threads(threads)
            cpu["single_core"] = {"value": ups1, "unit": UNIT, "cores": 1,
                                  "sample": "%d time step(s) of the full grid, %.1f s" % (nst1, secs1)}

    extras = None
    if world == 1 and args.workload == "dubinscar4d" and not args.no_extras:
        extras = extra_workloads(args)
    alu = {"bound": "alu", "achieved": alu_ops_per_node_step(problem) * N * steps_per_solve / (ms_per_step / 1000.0),
           "peak": GB300_FP32_LANE_OPS, "unit": "FP32 lane ops/s",
           "frac": alu_ops_per_node_step(problem) * N * steps_per_solve / (ms_per_step / 1000.0) / GB300_FP32_LANE_OPS,
           "ops_per_node_step": alu_ops_per_node_step(problem)}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": problem.name, "nodes": N, "time_steps_per_solve": steps_per_solve,
                       "scheme": "ENO%d + %s" % (problem.space_order,
                                                  "TVD-RK2" if problem.time_order == 2 else "Euler"),
                       "set": problem.set_kind, "cfl": problem.cfl, "horizon": problem.tau[-1],
                       "l2": "working set (%.0f MB) larger than L2 (129 MB)" % (
                           (16.0 if problem.obstacle is not None else 12.0) * N / 1e6),
                       "reach_avoid": problem.obstacle is not None,
                       "dissipation": problem.dissipation,
                       "parallelism": "independent solve per GPU",
                       "time_loop": "host-stepped" if args.host_loop else "one CUDA graph"},
            "gpu_launches": launches_per_solve * args.steps,
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "clocks": clocks,
            "alg_bytes_per_solve": bytes_per_solve,
            "solves_per_s": world * 1000.0 / ms_per_step,
            "roofline_alu": alu,
            "stage_pass": {"plane": "plane-streaming", "bulk": "bulk-staged"}.get(
                args.stage_pass, "plane-streaming" if problem.ndim < 4 else "bulk-staged"),
            "extra_workloads": extras,
        }
        print(json.dumps(line), flush=True)
    grid.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


def run_ttr(args):
    """Time-to-reach sweeping (Algorithm 2): one benchmark step is one complete
    solve (every sweep until the change drops to eps = 1e-5)."""
    import numpy as np
    import torch

    from paper_2204_05520_gb300 import _build, inputs, odp

    rank, world, local = rank_info()
    torch.cuda.set_device(local)
    dist = dist_setup(world, True)
    _build.build()
    odp.load()
    device = torch.device("cuda", local)
    problem = inputs.workload(args.workload)
    N = problem.points
    l_host = problem.target_values()
    stream = torch.cuda.Stream()
    l_dev = torch.from_numpy(l_host).to(device)
    grid = odp.Grid.for_problem(problem, stream=stream)
    if args.host_loop:
        odp.set_loop_mode(grid.handle, True)
    odp.set_stage_pass(grid.handle, {"auto": 0, "plane": 1, "bulk": 2}[args.stage_pass])
    grid.set_target(l_dev)
    st = None
    for _ in range(max(1, args.warmup)):
        st = grid.solve_ttr(stats=True)
    sweeps = int(st["sweeps"])
    sampler = ClockSampler(local)
    torch.cuda.synchronize()
    barrier(dist)
    sampler.start()
    time.sleep(0.3)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        grid.solve_ttr()
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier(dist)
    clocks = sampler.stop()
    ms_total = max_over_ranks(dist, ev0.elapsed_time(ev1), device)
    last = odp.solve_status(grid.handle)   # raises if the device flagged an error
    ms_per_step = ms_total / args.steps
    value = world * N * sweeps / (ms_per_step / 1000.0)
    peak, peak_kind = hbm_peak()
    alg_bytes = float(st["bytes"])
    achieved = alg_bytes / (ms_per_step / 1000.0) / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": None,
                "kernel": "k_ttr_tiles (whole sweep loop timed)", "peak_source": peak_kind,
                "alg_bytes_per_launch": alg_bytes / (sweeps * int(st["tile_planes"])),
                "avg_launch_ms": ms_per_step / (sweeps * int(st["tile_planes"])),
                "note": "the sweep is bounded by its serial hyperplane depth, not by bandwidth"}
    e2e = None
    if not args.no_e2e:
        l_pin = torch.from_numpy(l_host).pin_memory()
        out_pin = torch.empty_like(l_pin).pin_memory()
        torch.cuda.synchronize()
        barrier(dist)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            grid.set_target(l_pin)
            grid.solve_ttr()
            grid.readback(out_pin)
        t_e2e = max_over_ranks(dist, time.perf_counter() - t0, device)
        e2e = {"value": world * N * sweeps * args.steps / t_e2e, "unit": UNIT,
               "h2d_bytes_per_step": 4 * N, "d2h_bytes_per_step": 4 * N,
               "ms_per_step": 1000.0 * t_e2e / args.steps}
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        want = max(1, min(sweeps, int(2e8 // N)))
        ups, secs, threads, nsw = oracle_ttr_sample(problem, want)
        cpu = {"value": ups, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": "%d sweeps of the full %s grid (%d nodes), %.1f s" % (nsw, problem.name, N, secs)}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": problem.name, "nodes": N, "method": "Lax-Friedrichs sweeping",
                       "order": "Gauss-Seidel, alternating directions, hyperplane wavefronts",
                       "sweeps_per_solve": sweeps, "eps": 1e-5, "big": 1e4,
                       "tile_planes_per_sweep": int(st["tile_planes"]),
                       "l2": "working set (%.0f MB)%s L2 (129 MB)" % (
                           8.0 * N / 1e6, " larger than" if 8.0 * N > 129e6 else " inside"),
                       "parallelism": "independent solve per GPU",
                       "sweep_loop": "host-stepped" if args.host_loop else "one CUDA graph"},
            "gpu_launches": int(st["launches"]) * args.steps + args.steps,
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "clocks": clocks,
            "solve_ms": ms_per_step,
        }
        print(json.dumps(line), flush=True)
    grid.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


def measure_batch(steps, warmup, dist=None, local=0):
    """512 independent Dubins3D BRT solves (seed 0): one batched call against
    the same solves issued one at a time through grids created beforehand
    (no allocation in either timed region).  Returns a dict of figures."""
    import torch

    from paper_2204_05520_gb300 import inputs, odp

    problems = inputs.batch_problems(count=512, seed=0)
    stream = torch.cuda.Stream()
    grids = []
    for p in problems:
        g = odp.Grid.for_problem(p, stream=stream)
        g.set_target(torch.from_numpy(p.target_values()).cuda())
        grids.append(g)
    horizons = [p.tau[-1] for p in problems]
    for _ in range(warmup):
        st = odp.batch_solve(grids, horizons)
    torch.cuda.synchronize()
    barrier(dist)
    t0 = time.perf_counter()
    dev_ms = 0.0
    for _ in range(steps):
        st = odp.batch_solve(grids, horizons)
        dev_ms += st["device_ms"]
    batched_s = max_over_ranks(dist, (time.perf_counter() - t0) / steps, torch.device("cuda", local))
    # one at a time through the single-solve graph of each (pre-created) grid
    for g, p in zip(grids, problems):
        g.solve_problem(p)
    torch.cuda.synchronize()
    reps = max(1, steps // 5)
    t0 = time.perf_counter()
    for _ in range(reps):
        for g, p in zip(grids, problems):
            g.solve_problem(p)
        torch.cuda.synchronize()
    single_s = max_over_ranks(dist, (time.perf_counter() - t0) / reps, torch.device("cuda", local))
    n = len(problems)
    dev_s = dev_ms / steps / 1000.0
    out = {"solves": n, "nodes": sum(p.points for p in problems), "rounds": st["rounds"],
           "batched_s": batched_s, "batched_solves_per_s": n / batched_s,
           "device_ms_per_batch": 1000.0 * dev_s, "point_updates_per_s": st["point_updates"] / batched_s,
           "launches_per_batch": st.get("launches"), "tuned": st.get("tuned"),
           "one_at_a_time_solves_per_s": n / single_s, "one_at_a_time_s": single_s,
           "speedup_vs_one_at_a_time": single_s / batched_s,
           "roofline_frac": st["bytes"] / dev_s / 1e9 / hbm_peak()[0]}
    for g in grids:
        g.close()
    return out


def run_batch(args):
    import torch

    from paper_2204_05520_gb300 import _build, odp

    rank, world, local = rank_info()
    torch.cuda.set_device(local)
    dist = dist_setup(world, True)
    _build.build()
    odp.load()
    b = measure_batch(args.steps, args.warmup, dist, local)
    if rank == 0:
        line = {
            "metric": "batched solves/s", "value": world * b["batched_solves_per_s"], "unit": "solves/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * b["batched_s"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "batch512_dubins3d", "solves": b["solves"], "nodes": b["nodes"],
                       "rounds": b["rounds"]},
            "point_updates_per_s": b["point_updates_per_s"],
            "device_ms_per_batch": b["device_ms_per_batch"],
            "one_at_a_time": {"solves_per_s": b["one_at_a_time_solves_per_s"], "s_per_batch": b["one_at_a_time_s"]},
            "speedup_vs_one_at_a_time": b["speedup_vs_one_at_a_time"],
            "roofline": {"bound": "hbm", "frac": b["roofline_frac"], "peak": hbm_peak()[0], "unit": "GB/s"},
        }
        print(json.dumps(line), flush=True)
    return 0


def measure_served(rates, window, budget_gb, max_resident_mnodes=0.0, single_count=24):
    """Poisson request streams (seed 1) of Dubins3D and DubinsCar4D solves
    served with continuous batching under an HBM budget; p50/p99 latency
    (arrival -> result ready) and completed solves/s per arrival rate, and
    the same requests solved one at a time through grids created before the
    timed region.  Returns (points, one_at_a_time_solves_per_s)."""
    import numpy as np
    import torch

    from paper_2204_05520_gb300 import inputs, odp

    stream = torch.cuda.Stream()
    points = []
    budget = int(budget_gb * (1 << 30))
    with odp.Server(budget, stream=stream) as srv:
        srv.set_max_resident(int(max_resident_mnodes * 1e6))
        for rate in rates:
            count = int(min(2000, max(10, rate * window)))
            stream_reqs = inputs.served_requests(rate, count=count, seed=1)
            targets = [p.target_values() for _, p in stream_reqs]
            outs = {}
            lat, ids, arrival = [], {}, {}
            t0 = time.monotonic()
            nxt = 0
            done = 0
            deadline = t0 + 20.0 + window
            while done < count and time.monotonic() < deadline:
                now = time.monotonic() - t0
                while nxt < count and stream_reqs[nxt][0] <= now:
                    rid = srv.submit(stream_reqs[nxt][1], target=targets[nxt])
                    ids[rid] = nxt
                    arrival[rid] = t0 + stream_reqs[nxt][0]
                    nxt += 1
                if not ids:
                    time.sleep(min(0.002, max(0.0, stream_reqs[nxt][0] - now)))
                    continue
                srv.step(rounds=8)
                for rid in list(ids):
                    st = srv.poll(rid)
                    if st["state"] >= odp.REQ_DONE:
                        p = stream_reqs[ids[rid]][1]
                        out = outs.setdefault(p.n, np.empty(p.n, np.float32))
                        srv.readback(rid, out)
                        lat.append(st["t_done"] - arrival[rid])
                        srv.release(rid)
                        del ids[rid]
                        done += 1
            span = time.monotonic() - t0
            for rid in list(ids):
                try:
                    srv.release(rid)
                except odp.OdpError:
                    pass
            lat_sorted = sorted(lat)
            pct = lambda q: lat_sorted[min(len(lat_sorted) - 1, int(q * len(lat_sorted)))] if lat_sorted else None
            points.append({"rate": rate, "requests": count, "completed": done,
                           "solves_per_s": done / span if span > 0 else None,
                           "p50_s": pct(0.50), "p99_s": pct(0.99)})
            # drain anything still resident before the next rate
            while srv.info()["resident"] or srv.info()["queued"]:
                srv.step(rounds=64)
    # one at a time: requests of the same stream, each solved through its own
    # grid created (and given its target) before the timed region, result read
    # back to the host
    reqs = [p for _, p in inputs.served_requests(rates[-1], count=single_count, seed=1)]
    grids = []
    for p in reqs:
        g = odp.Grid.for_problem(p, stream=stream)
        g.set_target(p.target_values())
        grids.append(g)
    outs = [np.empty(p.n, np.float32) for p in reqs]
    grids[0].solve_problem(reqs[0])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for g, p, o in zip(grids, reqs, outs):
        g.solve_problem(p)
        g.readback(o)
    single = len(reqs) / (time.perf_counter() - t0)
    for g in grids:
        g.close()
    return points, single


def run_served(args):
    import torch

    from paper_2204_05520_gb300 import _build, odp

    rank, world, local = rank_info()
    torch.cuda.set_device(local)
    _build.build()
    odp.load()
    rates = [float(r) for r in args.rates.split(",")]
    points, single = measure_served(rates, args.window, args.budget_gb, args.max_resident_mnodes)
    best = max((pt["solves_per_s"] or 0.0) for pt in points)
    if rank == 0:
        line = {"metric": "served solves/s (saturation) with p50/p99 latency", "value": best,
                "unit": "solves/s", "n_gpus": 1, "steps": len(points), "warmup": 0,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic",
                "config": {"workload": "served_poisson_dubins3d_dubinscar4d", "budget_gb": args.budget_gb,
                           "window_s": args.window, "rounds_per_launch": 8,
                           "max_resident_nodes": int(args.max_resident_mnodes * 1e6)},
                "rates": points, "one_at_a_time_solves_per_s": single,
                "speedup_vs_one_at_a_time": best / single if single else None}
        print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch512":
        return run_batch(args)
    if args.workload == "served":
        return run_served(args)
    if args.workload in TTR_WORKLOADS:
        return run_ttr(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
