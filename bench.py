"""Benchmark: implicit time steps per second of the 2-D PFC 512x512 workload.

Workload (``pfc512``): periodic 512x512 grid, h = pi/(2 sqrt 3), eps = 0.4
(alpha = 0.6), gamma = 2, supercooled liquid rho = 0.80 with four seeded
Gaussian nuclei (amplitude 0.5) and 0.01 U(-1,1) noise, u = 0, s = 0.02,
FAS V(2,2) to a float64 residual of 1e-10, undamped point-block smoother.
The headline arm is the mixed path (float32 smoothing inside the float64
outer residual loop); the plain float64 path is timed beside it.  Each step
starts from the linear extrapolation in time of the last two converged
iterates (fm_params.init; --init previous starts from the previous time
level, which is also timed beside the headline); every step is solved to the
same float64 tolerance either way.

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
import platform
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "implicit steps/s at 512^2 (FP32-smoothed FAS, float64 residual 1e-10)"

# Algorithmic float32 words per grid point of one smoother sweep (the method's
# traffic): read the unknowns, the right-hand sides and the coefficients
# rho^k, omega^k once, write the unknowns once.
SWEEP_WORDS = {"pfc2d": 17, "cdft2d": 11, "pfc3d": 22}
UNIT = "steps/s"
WORKLOAD = "pfc512: 2-D PFC 512x512, eps=0.4, s=0.02, 4 nuclei, undamped, V(2,2) to 1e-10"


def rank_seed(rank):
    """Seed of the independent instance a rank advances."""
    return 2 + 1000 * rank


def shard(n, rank, world):
    """Instances of an ensemble of n that rank `rank` of `world` owns."""
    return list(range(rank, n, world))


def max_over_ranks(dist, value, device):
    """Largest value over all ranks (the job time is the slowest rank's)."""
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world, units_per_rank, max_ms):
    """Whole-job units per second: all ranks' units over the slowest rank's time."""
    return world * units_per_rank / (max_ms / 1e3)


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


def sweeps_per_launch(variant):
    """Red-black sweeps one launch of fused-sweep variant `variant` runs."""
    if variant in (34, 35):
        return 2
    if variant >= 30:
        return 1 + ((variant - 30) & 1)
    return 1 if variant == 28 else (2 if variant >= 18 else 1)


def sweep_kernel(variant, batched):
    """Name of the fused-sweep kernel that variant `variant` launches."""
    pre = "kb_" if batched else "k_"
    if variant == 34 and not batched:
        return ("k_smooth_coop<float,PFC> (a smoothing step's red and black passes in one cooperative launch, "
                "grid barriers between passes, in place)")
    if variant == 35 and not batched:
        return "k_smooth_rb2d<float,PFC,32x14> (two sweeps per launch, halo 4)"
    if variant in (34, 35):
        variant = 24
    if variant >= 30:
        if batched:  # the batch runs the small tiles as 0 and 24
            variant = 24 if variant & 1 else 0
        else:
            tile = "16x16" if variant < 32 else "16x8"
            return (f"k_smooth_rb2d<float,PFC,{tile}> ("
                    + ("two sweeps per launch, halo 4)" if variant & 1 else "one sweep per launch)"))
    if variant >= 27 and not batched:
        tile, ns = [("32x16", 2), ("32x16", 1), ("32x32", 2)][variant - 27]
        return (f"k_smooth_rb2d_tma<float,PFC,{tile}> (tile staged by tensor copies, "
                + ("two sweeps per launch, halo 4)" if ns == 2 else "one sweep per launch)"))
    if variant >= 27:  # the batch runs the tensor-copy variants as their cp.async twins
        variant = {27: 24, 28: 0, 29: 26}[variant]
    if variant >= 24:
        tile = ["32x16", "64x8", "32x32"][variant - 24]
        return f"{pre}smooth_rb2d<float,PFC,{tile}> (two sweeps per launch, halo 4)"
    if variant >= 12:
        m = (variant - 12) % 6
        tx = 64 if m < 3 else 128
        ly = 16 << (m % 3)
        if variant >= 18:
            return f"{pre}smooth_march2<float,PFC,{tx}> ({ly} rows per block, two sweeps per launch)"
        return f"{pre}smooth_march<float,PFC,{tx}> ({ly} rows per block)"
    tile = ["32x16", "64x8", "32x32"][variant >> 2]
    return (f"{pre}smooth_rb2d<float,PFC,{tile}> (f staged: {bool(variant & 2)}, "
            f"persistent: {bool(variant & 1)})")


def profiled_traffic(key, variant):
    """DRAM bytes per launch of fused-sweep variant `variant` from the
    committed ncu capture (profiles/traffic.json), or None when that variant
    has not been captured."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            ent = json.load(f).get(key)
    except (OSError, ValueError):
        return None
    if not ent:
        return None
    return ent.get("per_variant", {}).get(str(variant))


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "of measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "of fallback"


INIT = {"previous": 0, "extrapolate": 1}


def make_solver(fm, rho_shape, prm, precision, stream, init="previous", coarse=None):
    n = list(reversed(rho_shape))
    from paper_1503_07416_gb300 import inputs
    kw = {} if coarse is None else {"coarse_precision": coarse}
    return fm.Solver("pfc", n, prm["h"], alpha=prm["alpha"], precision=precision, tol=prm["tol"],
                     w_damp=0.0, gamma=prm["gamma"], delta=0.0, stream=stream, init=INIT[init],
                     **inputs.BENCH_MG_2D, **kw)


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

    rho, vel, prm = inputs.pfc512(seed=rank_seed(rank))
    N = rho.size
    stream = torch.cuda.current_stream().cuda_stream
    rho_d = torch.from_numpy(rho).cuda()
    vel_d = [torch.from_numpy(v).cuda() for v in vel]
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MiB > L2

    results = {}
    tuning = {}
    arms = [("mixed", fm.FM_MIXED, args.init, None), ("fp64", fm.FM_FP64, args.init, None)]
    if args.init != "previous":  # the same arm from the previous time level
        arms.append(("mixed_previous", fm.FM_MIXED, "previous", None))
    # the mixed arm with the coarsest-grid solve in float32 instead of float64
    arms.append(("mixed_coarse32", fm.FM_MIXED, args.init, fm.FM_MIXED))
    if args.only:
        arms = [a for a in arms if a[0] == args.only]
    for name, prec, init, coarse in arms:
        sol = make_solver(fm, rho.shape, prm, prec, stream, init, coarse)
        tuning[name] = [fm.fm_tuning(sol.handle, l) for l in range(3)]
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        with ClockSampler(local) as clk:
            times, cycles, launches = time_device_steps(
                torch, fm, sol, rho_d, vel_d, prm["dt"], args.steps, args.warmup, flush)
        prof = time_smoother(torch, fm, sol, rho_d, vel_d, prm["dt"], min(args.steps, 20), flush)
        total_ms = sum(times)
        if world > 1:
            total_ms = max_over_ranks(dist, total_ms, "cuda")
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

    # end to end through the C ABI with host buffers (mixed path): fm_step_host
    # copies the pinned inputs in, steps, and copies the new fields out
    sol = results["mixed"]["sol"]
    h_rho = torch.from_numpy(rho).pin_memory()
    h_vel = [torch.from_numpy(v).pin_memory() for v in vel]
    o_rho = torch.empty_like(h_rho).pin_memory()
    o_vel = [torch.empty_like(v).pin_memory() for v in h_vel]
    # two steppers in ping-pong (checked and marshalled once): each step's host
    # input is the previous step's host output, so the trajectory advances as
    # in the device-timed loop
    steppers = (sol.host_stepper(h_rho, h_vel, o_rho, o_vel), sol.host_stepper(o_rho, o_vel, h_rho, h_vel))
    for k in range(args.warmup):
        steppers[k & 1](prm["dt"])
    h_rho.copy_(torch.from_numpy(rho))
    for hv, v in zip(h_vel, vel):
        hv.copy_(torch.from_numpy(v))
    sol.set_fields(h_rho, h_vel)  # the timed steps start from the workload's state, history cleared
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    t0 = time.perf_counter()
    e_start = torch.cuda.Event(enable_timing=True)
    e_end = torch.cuda.Event(enable_timing=True)
    e_start.record()
    for k in range(args.steps):
        steppers[k & 1](prm["dt"])
    e_end.record()
    torch.cuda.synchronize()
    e2e_ms = e_start.elapsed_time(e_end)
    if world > 1:
        e2e_ms = max_over_ranks(dist, e2e_ms, "cuda")

    for r in results.values():
        r["sol"].close()

    peak, peak_kind = load_peaks()
    sec_batch = None
    if not args.no_secondary:
        # every rank steps its shard of the ensemble
        sec_batch = secondary_batch48(torch, fm, inputs, flush, peak, dist=dist, rank=rank, world=world)

    if rank != 0:
        dist.destroy_process_group() if world > 1 else None
        return

    mix, f64 = results["mixed"], results["fp64"]
    steps = args.steps
    value = job_throughput(world, steps, mix["total_ms"])
    ms_per_step = mix["total_ms"] / steps
    # smoother roofline: one launch of the fused 2-D kernel runs one (or, for
    # the two-sweep variants, two) red-black sweeps of the finest level and
    # moves the same algorithmic bytes either way: 20 words/point x N points
    # (float32): read e (5), f (5), rho^k, omega^k, rho, u, v (5); write e (5)
    sm_ms, sm_n = mix["prof"]
    spl = sweeps_per_launch(tuning["mixed"][0][0])
    words = 20
    bytes_launch = words * 4 * N
    avg_ms = sm_ms / max(1, sm_n)
    # the method's bytes: 17 float32 words per point per sweep (read 5
    # unknowns, 5 right-hand sides, rho^k, omega^k; write 5), times the sweeps
    # one launch runs
    bytes_method = SWEEP_WORDS["pfc2d"] * 4 * N * spl
    achieved = bytes_method / (avg_ms * 1e-3) / 1e9 if sm_n else None
    achieved_launch = bytes_launch / (avg_ms * 1e-3) / 1e9 if sm_n else None
    traffic = profiled_traffic("k_smooth_pfc512_level0", tuning["mixed"][0][0])
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
        "dtype": "f32 smoothing and transfers / f64 residual, coarsest solve, norms",
        "data": "synthetic (seeded)",
        "config": {
            "workload": WORKLOAD,
            "grid": [512, 512],
            "precision": "mixed",
            "l2": "flushed (256 MiB write) between timed steps, flush untimed",
            "cycles_per_step_mean": round(statistics.mean(mix["cycles"]), 3),
            "multigrid": {"cycle": "V(2,2)", "levels": "512^2 .. 64^2 (4)", "coarsest_sweeps": 2,
                          "coarse_solve": "2 red-black sweeps of the 64^2 grid in float64 on float64 copies of "
                                          "the level: a conversion launch in, 4 colour launches of 32-thread "
                                          "blocks, a conversion launch out (the float32-coarse arm: one fused "
                                          "two-sweep launch)"},
            "parallelism": f"{world} independent instance(s), one per GPU",
            "initial_iterate": {"previous": "previous time level (rho^k, u^k, mu^0, kappa^0)",
                                "extrapolate": "linear extrapolation in time of the last two converged iterates "
                                               "(fm_params.init = FM_INIT_EXTRAPOLATE; the first timed step starts "
                                               "with the history of the warm-up steps cleared)"}[args.init],
            "fp64_path": {
                "value": round(world * steps / (f64["total_ms"] / 1e3), 3),
                "ms_per_step": round(f64["total_ms"] / steps, 5),
                "cycles_per_step_mean": round(statistics.mean(f64["cycles"]), 3),
                "smoother_launch_ms": round(f64_avg, 6),
                "smoother_sweeps_per_launch": sweeps_per_launch(tuning["fp64"][0][0]),
                "smoother_gbs": round(words * 8 * N / (f64_avg * 1e-3) / 1e9, 1) if f64_sm_n else None,
            },
            "speedup_mixed_over_fp64": round(f64["total_ms"] / mix["total_ms"], 3),
            "coarse_solve_precision": "float64 (fm_params.coarse_precision = FM_FP64)",
            "mixed_coarse_solve_float32": (
                {"value": round(world * steps / (results["mixed_coarse32"]["total_ms"] / 1e3), 3),
                 "cycles_per_step_mean": round(statistics.mean(results["mixed_coarse32"]["cycles"]), 3)}
                if "mixed_coarse32" in results else None),
            "mixed_from_previous_time_level": (
                {"value": round(world * steps / (results["mixed_previous"]["total_ms"] / 1e3), 3),
                 "cycles_per_step_mean": round(statistics.mean(results["mixed_previous"]["cycles"]), 3)}
                if "mixed_previous" in results else None),
            "sweep_variants": {k: [{"level": l, "variant": v[0], "ms": [round(x, 4) for x in v[1]]}
                                   for l, v in enumerate(vals)] for k, vals in tuning.items()},
        },
        "roofline": {
            "kernel": sweep_kernel(tuning["mixed"][0][0], False) + ", finest level",
            "sweeps_per_launch": spl,
            "bound": "hbm",
            "achieved": round(achieved, 1) if achieved else None,
            "peak": peak,
            "unit": "GB/s",
            "frac": round(achieved / peak, 4) if achieved else None,
            "frac_survey": round(achieved / peak, 4) if achieved else None,
            "peak_source": peak_kind,
            "traffic": traffic,
            "algorithmic_bytes_per_launch": bytes_method,
            "bytes_count": "17 float32 words per point per sweep x sweeps per launch (the method's traffic)",
            "per_launch_20_words": {
                "bytes": bytes_launch,
                "achieved": round(achieved_launch, 1) if achieved_launch else None,
                "frac": round(achieved_launch / peak, 4) if achieved_launch else None,
                "count": "20 float32 words per point per launch: the 17 plus the coefficient iterate "
                         "rho, u, v that the correction form reads"},
            "launch_ms": round(avg_ms, 6),
            "dof_sweeps_per_s": round(5 * N * spl / (avg_ms * 1e-3), 1) if sm_n else None,  # 5 unknowns/point
            "launches_timed": sm_n,
            "launch_timing": "CUDA events around each finest-level smoother launch, in a pass of "
                             "the same steps run launch by launch (the timed steps run as graphs)",
        },
        "e2e": {
            "value": round(job_throughput(world, steps, e2e_ms), 3),
            "unit": UNIT,
            "h2d_bytes_per_step": 3 * N * 8,
            "d2h_bytes_per_step": 3 * N * 8,
            "api": "fm_step_host (pinned host rho, u, v in; new rho, u, v out; one synchronisation per step)",
        },
        "gpu_launches": mix["launches"],
        "clocks": mix["clocks"],
    }
    if not args.no_secondary:
        out["secondary"] = dict(batch48=sec_batch, **secondary_all(torch, fm, inputs, flush, peak))
    if not args.no_cpu_baseline and world == 1:
        out["cpu_baseline"] = cpu_baseline(args.cpu_steps)
    print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()


def _timed_steps(torch, step_fn, steps, flush):
    """CUDA-event time (ms) of each call of step_fn, L2 flushed (untimed)
    before each."""
    stream = torch.cuda.current_stream()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    out = []
    for k in range(steps):
        flush.zero_()
        ev[k][0].record(stream)
        out.append(step_fn())
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in ev], out


def secondary_batch48(torch, fm, inputs, flush, peak, steps=3, warmup=2, dist=None, rank=0, world=1):
    """48 independent PFC instances (n from {128..1024}, per-instance dt),
    mixed precision, stepped together (fm_step_batch).  Under torchrun each
    rank steps its shard of the ensemble as one batch (instances are
    independent: no collective on the data path); the ensemble's time is the
    slowest rank's."""
    full = inputs.batch48()
    mine = shard(len(full), rank, world)
    ens = [full[i] for i in mine]
    sizes = [prm["n"] for _, _, prm in ens]
    p0 = ens[0][2]
    stream = torch.cuda.current_stream().cuda_stream
    b = fm.Batch("pfc", sizes, p0["h"], alpha=p0["alpha"], precision=fm.FM_MIXED, tol=p0["tol"],
                 w_damp=0.0, gamma=p0["gamma"], delta=0.0, stream=stream, **inputs.BENCH_MG_2D)
    for i, (rho, vel, _) in enumerate(ens):
        b.set_fields(i, rho, vel)
    dts = [prm["dt"] for _, _, prm in ens]
    for _ in range(warmup):
        b.step(dts)
    for i, (rho, vel, _) in enumerate(ens):
        b.set_fields(i, rho, vel)
    torch.cuda.synchronize()
    l0 = fm.fm_batch_launches(b.handle)
    if world > 1:
        dist.barrier()
    times, infos = _timed_steps(torch, lambda: b.step(dts), steps, flush)
    launches = fm.fm_batch_launches(b.handle) - l0
    ms_sm, pts = fm.fm_batch_time_smoother(b.handle, 20)
    tune0 = fm.fm_batch_tuning(b.handle, 0)
    one = None
    if sweeps_per_launch(tune0[0]) == 2:
        # the fastest one-sweep variant of the autotuner's table, timed the same way
        v1 = min((v for v in range(18) if tune0[1][v] > 0), key=lambda v: tune0[1][v])
        ms1, _ = fm.fm_batch_time_sweep_variant(b.handle, v1, 20)
        g1 = SWEEP_WORDS["pfc2d"] * 4 * pts / (ms1 * 1e-3) / 1e9
        one = {"kernel": sweep_kernel(v1, True), "variant": v1, "launch_ms": round(ms1, 5),
               "achieved": round(g1, 1), "frac": round(g1 / peak, 4), "frac_survey": round(g1 / peak, 4),
               "frac_20_words": round(g1 * 20 / SWEEP_WORDS["pfc2d"] / peak, 4),
               "dof_sweeps_per_s": round(5 * pts / (ms1 * 1e-3), 1),
               "traffic": profiled_traffic("kb_smooth_batch48", v1)}
    b.close()
    cyc = [i.cycles for inf in infos for i in inf]
    total = sum(times)
    if world > 1:
        total = max_over_ranks(dist, total, "cuda")
    spl = sweeps_per_launch(tune0[0])
    gbs = SWEEP_WORDS["pfc2d"] * 4 * pts * spl / (ms_sm * 1e-3) / 1e9
    return {
        "workload": "batch48: 48 PFC instances, n in {128,256,512,1024}, dt log-uniform [1e-3,1e-1], "
                    "eps=0.4, mixed, V(2,2) to 1e-10",
        "points": int(sum(prm["n"] ** 2 for _, _, prm in full)),
        "ranks": world,
        "instances_on_rank0": len(sizes),
        "instance_steps_per_s": round(len(full) * steps / (total / 1e3), 2),
        "batch_steps_per_s": round(steps / (total / 1e3), 3),
        "ms_per_batch_step": round(total / steps, 3),
        "cycles_mean": round(sum(cyc) / len(cyc), 3), "cycles_max": max(cyc),
        "gpu_launches": launches,
        "smoother_roofline": {"kernel": sweep_kernel(tune0[0], True) + ", finest level of all instances",
                              "bound": "hbm", "achieved": round(gbs, 1), "peak": peak, "unit": "GB/s",
                              "frac": round(gbs / peak, 4), "frac_survey": round(gbs / peak, 4),
                              "frac_20_words_per_launch": round(20 * 4 * pts / (ms_sm * 1e-3) / 1e9 / peak, 4),
                              "bytes_count": "17 float32 words per point per sweep x sweeps per launch",
                              "launch_ms": round(ms_sm, 5),
                              "sweeps_per_launch": spl,
                              "dof_sweeps_per_s": round(5 * pts * sweeps_per_launch(tune0[0]) / (ms_sm * 1e-3),
                                                        1),
                              "algorithmic_bytes_per_launch": SWEEP_WORDS["pfc2d"] * 4 * pts * spl,
                              "timing": "20 back-to-back launches after a warm-up, CUDA events",
                              "traffic": profiled_traffic("kb_smooth_batch48", tune0[0]),
                              "autotuned_variant": tune0[0],
                              "variant_ms": [round(x, 4) for x in tune0[1]],
                              # a two-sweep launch moves one pass of bytes for two sweeps; the best
                              # one-sweep kernel shows the HBM fraction of a single sweep
                              "one_sweep": one},
    }


def smoother_sweeps_per_launch(fm, sol, dim):
    """Red-black sweeps one finest-level smoother launch runs: the fused 2-D
    variants run one or two; the 3-D smoother's variant is reported by
    fm_tuning too (see sweeps_per_launch_3d)."""
    v = fm.fm_tuning(sol.handle, 0)[0]
    return sweeps_per_launch_3d(v) if dim == 3 else sweeps_per_launch(v)


def sweeps_per_launch_3d(variant):
    """3-D smoother variants (fm_tuning): 0 and 1 run a red and a black launch
    per sweep (half a sweep per timed launch); 2 runs a sweep in z-chunks and
    its timing events bracket the whole sweep; 3 and 4 (z-marching) run one
    sweep per launch."""
    return 1 if variant >= 2 else 0.5


def secondary_single(torch, fm, flush, kind, rho, vel, prm, precision, steps, warmup=2, dim=2, smoother=False,
                     peak=None):
    n = list(reversed(rho.shape))
    stream = torch.cuda.current_stream().cuda_stream
    from paper_1503_07416_gb300 import inputs
    mg = inputs.BENCH_MG_2D if dim == 2 else {}
    sol = fm.Solver(kind, n, prm["h"], dim=dim, alpha=prm.get("alpha", 0.0), nu=prm.get("nu", 0.0),
                    precision=precision, tol=prm["tol"], w_damp=0.0,
                    delta=prm.get("delta", 0.0), gamma=prm["gamma"], stream=stream, **mg)
    rho_d = torch.from_numpy(rho).cuda()
    vel_d = [torch.from_numpy(v).cuda() for v in vel]
    sol.set_fields(rho_d, vel_d)
    for _ in range(warmup):
        sol.step(prm["dt"])
    sol.set_fields(rho_d, vel_d)
    torch.cuda.synchronize()
    times, infos = _timed_steps(torch, lambda: sol.step(prm["dt"]), steps, flush)
    out = {"steps_per_s": round(steps / (total_ms(times) / 1e3), 3), "ms_per_step": round(total_ms(times) / steps, 4),
           "cycles_mean": round(sum(i.cycles for i in infos) / len(infos), 3)}
    if smoother:
        ms, n = time_smoother(torch, fm, sol, rho_d, vel_d, prm["dt"], 2, flush)
        per = ms / max(1, n)
        spl = smoother_sweeps_per_launch(fm, sol, dim)
        key = "pfc3d" if dim == 3 else ("pfc2d" if kind == "pfc" else "cdft2d")
        wb = 4 if precision == fm.FM_MIXED else 8
        nu = (5 if kind == "pfc" else 3) + (1 if dim == 3 else 0)
        bytes_launch = SWEEP_WORDS[key] * wb * rho.size * spl
        gbs = bytes_launch / (per * 1e-3) / 1e9
        out["smoother"] = {"kernel_variant": fm.fm_tuning(sol.handle, 0)[0], "launch_ms": round(per, 5),
                           "sweeps_per_launch": spl, "launches_timed": n,
                           "dof_sweeps_per_s": round(nu * rho.size * spl / (per * 1e-3), 1),
                           "achieved_gbs": round(gbs, 1), "bound": "hbm", "unit": "GB/s", "peak": peak,
                           "frac": round(gbs / peak, 4) if peak else None,
                           "frac_survey": round(gbs / peak, 4) if peak else None,
                           "algorithmic_bytes_per_launch": bytes_launch,
                           "bytes_count": f"{SWEEP_WORDS[key]} words per point per sweep x sweeps per launch"}
    sol.close()
    return out


def total_ms(times):
    return sum(times)


def profile_batch(count):
    """Small ncu target: the first `count` instances of batch48, one step,
    then 4 timed finest-level batched sweeps."""
    import torch
    from paper_1503_07416_gb300 import build, fm, inputs
    build.build_library()
    ens = inputs.batch48()[:count]
    sizes = [prm["n"] for _, _, prm in ens]
    p0 = ens[0][2]
    b = fm.Batch("pfc", sizes, p0["h"], alpha=p0["alpha"], precision=fm.FM_MIXED, tol=p0["tol"], w_damp=0.0,
                 stream=torch.cuda.current_stream().cuda_stream, **inputs.BENCH_MG_2D)
    for i, (rho, vel, _) in enumerate(ens):
        b.set_fields(i, rho, vel)
    b.step([prm["dt"] for _, _, prm in ens])
    ms, pts = fm.fm_batch_time_smoother(b.handle, 4)
    torch.cuda.synchronize()
    b.close()
    print(json.dumps({"profile_batch": count, "points": pts, "ms_per_launch": ms,
                      "gbs": 80 * pts / (ms * 1e-3) / 1e9}))


def profile_single(name):
    """Small ncu target: one solver of a named workload (mixed), 1 warm-up and
    2 steps."""
    import torch
    from paper_1503_07416_gb300 import build, fm, inputs
    build.build_library()
    if name in ("gradflow512", "nanocrystal256"):
        sol, rho, vel, dt, _ = model_solver(torch, fm, inputs, name)
        sol.set_fields(rho, vel)
        cyc = [sol.step(dt).cycles for _ in range(3)]
        torch.cuda.synchronize()
        sol.close()
        print(json.dumps({"profile_single": name, "cycles": cyc}))
        return
    rho, vel, prm = getattr(inputs, name)()
    n = list(reversed(rho.shape))
    sol = fm.Solver(prm["kind"], n, prm["h"], dim=prm["dim"], alpha=prm.get("alpha", 0.0), nu=prm.get("nu", 0.0),
                    precision=fm.FM_MIXED, tol=prm["tol"], w_damp=0.0, delta=prm.get("delta", 0.0),
                    stream=torch.cuda.current_stream().cuda_stream,
                    **(inputs.BENCH_MG_2D if prm["dim"] == 2 else {}))
    sol.set_fields(rho, vel)
    cyc = [sol.step(prm["dt"]).cycles for _ in range(3)]
    torch.cuda.synchronize()
    sol.close()
    print(json.dumps({"profile_single": name, "cycles": cyc}))


def secondary_model(torch, fm, inputs, flush, name, steps=20, warmup=3):
    """Steps/s of the two models beside the periodic hydrodynamic one: the
    gradient flow (FM_GRADFLOW) on the pfc512 state and the channel
    (FM_WALLS_Y) on the 256^2 nanocrystal with the walls at -0.1 / +0.1;
    mixed precision, V(2,2) to 1e-10."""
    sol, rho, vel, dt, desc = model_solver(torch, fm, inputs, name)
    rho_d = torch.from_numpy(rho).cuda()
    vel_d = [torch.from_numpy(v).cuda() for v in vel] if vel is not None else None
    sol.set_fields(rho_d, vel_d)
    for _ in range(warmup):
        sol.step(dt)
    sol.set_fields(rho_d, vel_d)
    torch.cuda.synchronize()
    l0 = fm.fm_profile_read(sol.handle)[2]
    times, infos = _timed_steps(torch, lambda: sol.step(dt), steps, flush)
    launches = fm.fm_profile_read(sol.handle)[2] - l0
    sol.close()
    return {"workload": desc, "steps_per_s": round(steps / (sum(times) / 1e3), 3),
            "ms_per_step": round(sum(times) / steps, 4),
            "cycles_mean": round(sum(i.cycles for i in infos) / len(infos), 3), "gpu_launches": launches}


def model_solver(torch, fm, inputs, name):
    stream = torch.cuda.current_stream().cuda_stream
    if name == "gradflow512":
        rho, _, prm = inputs.pfc512()
        sol = fm.Solver("pfc", (512, 512), prm["h"], alpha=prm["alpha"], precision=fm.FM_MIXED, tol=1e-10,
                        w_damp=0.3, model=fm.FM_GRADFLOW, max_cycles=200, stream=stream, **inputs.BENCH_MG_2D)
        return sol, rho, None, 0.02, ("gradflow512: PFC gradient flow (Thm 3.3) from the pfc512 state, s = 0.02, "
                                      "w = 0.3 (the damping this sixth-order flow converges fastest with), mixed, "
                                      "V(2,2) to 1e-10, the benchmark hierarchy (coarsest 64, 2 coarse sweeps)")
    rho, vel, prm = inputs.nanocrystal(256)
    sol = fm.Solver("pfc", (256, 256), prm["h"], alpha=prm["alpha"], precision=fm.FM_MIXED, tol=1e-10, w_damp=0.0,
                    walls=fm.FM_WALLS_Y, u_wall=(-0.1, 0.1), max_cycles=200, stream=stream, **inputs.BENCH_MG_2D)
    return sol, rho, vel, prm["dt"], ("nanocrystal256: 2-D PFC channel (walls at -0.1/+0.1), hexagonal seed, "
                                      "eps = 0.4, s = 0.02, mixed, V(2,2) to 1e-10, the benchmark hierarchy")


def secondary_all(torch, fm, inputs, flush, peak):
    out = {"gradflow512": secondary_model(torch, fm, inputs, flush, "gradflow512"),
           "nanocrystal256": secondary_model(torch, fm, inputs, flush, "nanocrystal256")}
    rho, vel, prm = inputs.cdft256()
    out["cdft256"] = {
        "workload": "cdft256: 2-D CDFT 256x256, h=17/128, nu=2.362, s=0.02, delta 1e-10, undamped, V(2,2) to 1e-10",
        "mixed": secondary_single(torch, fm, flush, "cdft", rho, vel, prm, fm.FM_MIXED, 20, smoother=True, peak=peak),
        "fp64": secondary_single(torch, fm, flush, "cdft", rho, vel, prm, fm.FM_FP64, 10),
    }
    rho, vel, prm = inputs.pfc3d128()
    out["pfc3d128"] = {
        "workload": "pfc3d128: 3-D PFC 128^3, eps=0.4, s=0.02, one nucleus, undamped, V(2,2) to 1e-10",
        "mixed": secondary_single(torch, fm, flush, "pfc", rho, vel, prm, fm.FM_MIXED, 5, dim=3, smoother=True,
                                  peak=peak),
        "fp64": secondary_single(torch, fm, flush, "pfc", rho, vel, prm, fm.FM_FP64, 2, warmup=1, dim=3),
    }
    return out


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


def host_info():
    """Core count and CPU model of the host the oracle runs on."""
    model = platform.processor() or platform.machine()
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                key = line.split(":")[0].strip().lower()
                if key in ("model name", "cpu part", "hardware"):
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    return {"nproc": os.cpu_count(), "cpu": model, "machine": platform.machine()}


def cpu_baseline(nsteps):
    done, dt = oracle_steps(nsteps, 30.0)
    return {"value": round(done / dt, 5), "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{done} steps of the pfc512 workload (numpy FP64 oracle, single thread)",
            "host": host_info()}


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
                         "sample": f"{done} steps of the pfc512 workload (bounded to ~120 s)",
                         "host": host_info()},
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
    ap.add_argument("--only", choices=["mixed", "fp64", "mixed_previous", "mixed_coarse32"], default=None,
                    help="time one arm only and print a short diagnostic line (profiling runs)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--profile-single", choices=["pfc512", "cdft256", "pfc3d128", "pfc64", "gradflow512",
                                                 "nanocrystal256"], default=None,
                    help="profiling target: one solver of the named workload, 3 steps")
    ap.add_argument("--profile-batch", type=int, default=0,
                    help="profiling target: first K batch48 instances, timed batched sweeps only")
    ap.add_argument("--init", choices=list(INIT), default="extrapolate",
                    help="initial iterate of each step of the 512^2 arms")
    ap.add_argument("--no-secondary", action="store_true",
                    help="skip the batched, CDFT and 3-D workloads measured beside the headline")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.profile_batch:
        profile_batch(args.profile_batch)
    elif args.profile_single:
        profile_single(args.profile_single)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
