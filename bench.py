"""Benchmark: implicit time steps per second of the 2-D PFC 512x512 workload.

Workload (``pfc512``): periodic 512x512 grid, h = pi/(2 sqrt 3), eps = 0.4
(alpha = 0.6), gamma = 2, supercooled liquid rho = 0.80 with four seeded
Gaussian nuclei (amplitude 0.5) and 0.01 U(-1,1) noise, u = 0, s = 0.02,
FAS V(2,2) to a float64 residual of 1e-10, undamped point-block smoother.
The headline arm is the mixed path (float32 smoothing inside the float64
outer residual loop); the plain float64 path is timed beside it.

One "step" = one fm_step (the whole hot path: vorticity, source, the FAS
solve to tolerance, closure).  Inputs are resident in HBM when the timed
region starts; L2 is flushed (a 256 MiB write) between timed steps and the
flush is outside the per-step CUDA-event timing.  ``e2e`` times the same steps
through the C ABI with host buffers: each step copies rho, u, v from pinned
host memory in and the new rho, u, v back out.

``--impl reference`` times the FP64 CPU oracle on the same workload (a bounded
number of its steps) on the host cores.

Under torchrun each rank advances its own independent instance (weak scaling,
no collective on the data path); the timing is the max over ranks.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "implicit steps/s at 512^2 (FP32-smoothed FAS, float64 residual 1e-10)"
UNIT = "steps/s"
WORKLOAD = "pfc512: 2-D PFC 512x512, eps=0.4, s=0.02, 4 nuclei, V(2,2) to 1e-10"


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index),
                 "--query-gpu=clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
                 "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
                 "clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[3:7]):
                if val.lower() in ("active", "1"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "of measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "of fallback"


def make_solver(fm, rho_shape, prm, precision, stream):
    n = list(reversed(rho_shape))
    return fm.Solver("pfc", n, prm["h"], alpha=prm["alpha"], precision=precision, tol=prm["tol"],
                     w_damp=0.0, gamma=prm["gamma"], delta=0.0, stream=stream)


def time_device_steps(torch, fm, sol, rho_d, vel_d, dt, steps, warmup, flush):
    """Per-step CUDA-event times (ms) of `steps` fm_step calls (each one CUDA
    graph launch) on resident inputs, L2 flushed between steps (untimed);
    returns (times, cycles, kernels launched)."""
    stream = torch.cuda.current_stream()
    sol.set_fields(rho_d, vel_d)
    for _ in range(warmup):
        sol.step(dt)
    sol.set_fields(rho_d, vel_d)
    torch.cuda.synchronize()
    l0 = fm.fm_profile_read(sol.handle)[2]
    cycles = []
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for k in range(steps):
        flush.zero_()
        ev[k][0].record(stream)
        info = sol.step(dt)
        ev[k][1].record(stream)
        cycles.append(info.cycles)
    torch.cuda.synchronize()
    times = [a.elapsed_time(b) for a, b in ev]
    return times, cycles, fm.fm_profile_read(sol.handle)[2] - l0


def time_smoother(torch, fm, sol, rho_d, vel_d, dt, steps, flush):
    """CUDA-event duration of every finest-level smoother launch over `steps`
    steps of the same workload, run launch by launch (profiling mode: the
    events sit between the launches on the library's stream)."""
    sol.set_fields(rho_d, vel_d)
    torch.cuda.synchronize()
    fm.fm_profile(sol.handle, True)
    for _ in range(steps):
        flush.zero_()
        sol.step(dt)
    torch.cuda.synchronize()
    ms, n, _ = fm.fm_profile_read(sol.handle)
    fm.fm_profile(sol.handle, False)
    return ms, n


def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_1503_07416_gb300 import build, fm, inputs

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    if rank == 0 or world > 1:
        build.build_library()
    if world > 1:
        dist.barrier()
    fm.lib()

    rho, vel, prm = inputs.pfc512(seed=2 + 1000 * rank)
    N = rho.size
    stream = torch.cuda.current_stream().cuda_stream
    rho_d = torch.from_numpy(rho).cuda()
    vel_d = [torch.from_numpy(v).cuda() for v in vel]
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MiB > L2

    results = {}
    arms = (("mixed", fm.FM_MIXED), ("fp64", fm.FM_FP64))
    if args.only:
        arms = tuple(a for a in arms if a[0] == args.only)
    for name, prec in arms:
        sol = make_solver(fm, rho.shape, prm, prec, stream)
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        with ClockSampler(local) as clk:
            times, cycles, launches = time_device_steps(
                torch, fm, sol, rho_d, vel_d, prm["dt"], args.steps, args.warmup, flush)
        prof = time_smoother(torch, fm, sol, rho_d, vel_d, prm["dt"], min(args.steps, 20), flush)
        total_ms = sum(times)
        if world > 1:
            t = torch.tensor([total_ms], device="cuda", dtype=torch.float64)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            total_ms = float(t.item())
        results[name] = dict(total_ms=total_ms, cycles=cycles, launches=launches, prof=prof,
                             clocks=clk.summary(), sol=sol, prec=prec)

    if args.no_e2e or args.only:
        for r in results.values():
            r["sol"].close()
        if rank == 0:
            print(json.dumps({k: {"ms_per_step": v["total_ms"] / args.steps, "cycles": v["cycles"][:5],
                                  "launches": v["launches"], "smoother": v["prof"]}
                              for k, v in results.items()}))
        return

    # end to end through the C ABI with host buffers (mixed path)
    sol = results["mixed"]["sol"]
    h_rho = torch.from_numpy(rho).pin_memory()
    h_vel = [torch.from_numpy(v).pin_memory() for v in vel]
    o_rho = torch.empty_like(h_rho).pin_memory()
    o_vel = [torch.empty_like(v).pin_memory() for v in h_vel]
    for _ in range(args.warmup):
        sol.set_fields(h_rho, h_vel)
        sol.step(prm["dt"])
        sol.get_fields(o_rho, o_vel)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    t0 = time.perf_counter()
    e_start = torch.cuda.Event(enable_timing=True)
    e_end = torch.cuda.Event(enable_timing=True)
    e_start.record()
    for _ in range(args.steps):
        sol.set_fields(h_rho, h_vel)
        sol.step(prm["dt"])
        sol.get_fields(o_rho, o_vel)
    e_end.record()
    torch.cuda.synchronize()
    e2e_ms = e_start.elapsed_time(e_end)
    if world > 1:
        t = torch.tensor([e2e_ms], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_ms = float(t.item())

    for r in results.values():
        r["sol"].close()

    if rank != 0:
        dist.destroy_process_group() if world > 1 else None
        return

    mix, f64 = results["mixed"], results["fp64"]
    steps = args.steps
    value = world * steps / (mix["total_ms"] / 1e3)
    ms_per_step = mix["total_ms"] / steps
    peak, peak_kind = load_peaks()
    # smoother roofline: one launch of the fused 2-D kernel is one red-black
    # sweep of the finest level: algorithmic bytes = 20 words/point x N points
    # (float32): read e (5), f (5), rho^k, omega^k, rho, u, v (5); write e (5)
    sm_ms, sm_n = mix["prof"]
    words = 20
    bytes_launch = words * 4 * N
    avg_ms = sm_ms / max(1, sm_n)
    achieved = bytes_launch / (avg_ms * 1e-3) / 1e9 if sm_n else None
    traffic = None
    tpath = os.path.join(ROOT, "profiles", "smoother_traffic.json")
    if os.path.exists(tpath):
        try:
            traffic = json.load(open(tpath)).get("mixed_pfc512_bytes_per_launch")
        except (OSError, ValueError):
            traffic = None
    f64_sm_ms, f64_sm_n = f64["prof"]
    f64_avg = f64_sm_ms / max(1, f64_sm_n)
    out = {
        "metric": METRIC,
        "value": round(value, 3),
        "unit": UNIT,
        "n_gpus": world,
        "steps": steps,
        "warmup": args.warmup,
        "ms_per_step": round(ms_per_step, 5),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32 smoothing / f64 residual",
        "data": "synthetic (seeded)",
        "config": {
            "workload": WORKLOAD,
            "grid": [512, 512],
            "precision": "mixed",
            "l2": "flushed (256 MiB write) between timed steps, flush untimed",
            "cycles_per_step_mean": round(statistics.mean(mix["cycles"]), 3),
            "parallelism": f"{world} independent instance(s), one per GPU",
            "fp64_path": {
                "value": round(world * steps / (f64["total_ms"] / 1e3), 3),
                "ms_per_step": round(f64["total_ms"] / steps, 5),
                "cycles_per_step_mean": round(statistics.mean(f64["cycles"]), 3),
                "smoother_launch_ms": round(f64_avg, 6),
                "smoother_gbs": round(words * 8 * N / (f64_avg * 1e-3) / 1e9, 1) if f64_sm_n else None,
            },
            "speedup_mixed_over_fp64": round(f64["total_ms"] / mix["total_ms"], 3),
        },
        "roofline": {
            "kernel": "k_smooth_rb2d<float,PFC> (finest level, one red-black sweep)",
            "bound": "hbm",
            "achieved": round(achieved, 1) if achieved else None,
            "peak": peak,
            "unit": "GB/s",
            "frac": round(achieved / peak, 4) if achieved else None,
            "peak_source": peak_kind,
            "traffic": traffic,
            "algorithmic_bytes_per_launch": bytes_launch,
            "launch_ms": round(avg_ms, 6),
            "launches_timed": sm_n,
            "launch_timing": "CUDA events around each finest-level smoother launch, in a pass of "
                             "the same steps run launch by launch (the timed steps run as graphs)",
        },
        "e2e": {
            "value": round(world * steps / (e2e_ms / 1e3), 3),
            "unit": UNIT,
            "h2d_bytes_per_step": 3 * N * 8,
            "d2h_bytes_per_step": 3 * N * 8,
        },
        "gpu_launches": mix["launches"],
        "clocks": mix["clocks"],
    }
    if not args.no_cpu_baseline and world == 1:
        out["cpu_baseline"] = cpu_baseline(args.cpu_steps)
    print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()


def oracle_steps(nsteps, budget_s):
    """Time the FP64 CPU oracle on the pfc512 workload; at most nsteps steps or
    until budget_s seconds have elapsed (at least one step)."""
    from oracle import scheme as S
    from paper_1503_07416_gb300 import inputs
    rho, vel, prm = inputs.pfc512()
    P = S.Params(kind=S.PFC, dim=2, h=prm["h"], s=prm["dt"], alpha=prm["alpha"], gamma=prm["gamma"],
                 w_damp=0.0)
    opts = S.SolverOpts(tol=prm["tol"])
    done = 0
    t0 = time.perf_counter()
    while done < nsteps:
        rho, vel, _ = S.step(rho, vel, P, opts)
        done += 1
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    return done, dt


def cpu_baseline(nsteps):
    done, dt = oracle_steps(nsteps, 30.0)
    return {"value": round(done / dt, 5), "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{done} steps of the pfc512 workload (numpy FP64 oracle, single thread)"}


def run_reference(args):
    rank, world, local = dist_env()
    if rank != 0:
        return
    done, dt = oracle_steps(args.steps, 120.0)
    value = done / dt
    out = {
        "metric": METRIC, "value": round(value, 5), "unit": UNIT, "n_gpus": world,
        "steps": done, "warmup": 0, "ms_per_step": round(1e3 * dt / done, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded)", "impl": "reference",
        "config": {"workload": WORKLOAD, "grid": [512, 512], "precision": "fp64 oracle"},
        "cpu_baseline": {"value": round(value, 5), "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"{done} steps of the pfc512 workload (bounded to ~120 s)"},
        "e2e": {"value": round(value, 5), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-steps", type=int, default=4)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--only", choices=["mixed", "fp64"], default=None,
                    help="time one arm only and print a short diagnostic line (profiling runs)")
    ap.add_argument("--no-e2e", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
