"""The paper's experiments run through libfm (Sec. 6.1, Sec. 6.2).

``convergence``  Sec. 6.1.1 (CDFT) and Sec. 6.1.2 (PFC): the smooth initial
                 density of the paper on [0, 32)^2, zero velocity, evolved to
                 t_f = 10 along the refinement path s = 0.025 h^2 on grids
                 16^2, 32^2, ...; the Cauchy errors
                 e^{h;h/2}_{ij} = f^h_{ij} - f^{h/2}_{2i,2j} of rho, u and v,
                 their discrete L2 norms sqrt(h^2 sum e^2) (the coarse
                 spacing) and the rates log2(||e^{2h;h}|| / ||e^{h;h/2}||),
                 printed beside the paper's Tables 1-6.
``freezing``     Sec. 6.2: a supercooled liquid rho = rho_bar (1 + 0.1 eta)
                 freezing (CDFT: [0, 17)^2, 128^2, nu = 2.362, s = 0.02; PFC:
                 [0, 32)^2, 128^2, eps = 0.025, s = 0.01), one JSON record per
                 logged step with the energy components the paper plots
                 (KE, F and its parts: F_id / F_ex for CDFT, the four PFC
                 terms), the total energy E, the mass, the V-cycles and the
                 residual; E is checked to be non-increasing at every step.

Both run the float64 path of the CUDA library (the Cauchy errors of the fine
rungs, ~1e-9, are below what the float32-smoothed path guarantees per step).
Initial data come from ``inputs`` (seeded, synthetic).

    python -m paper_1503_07416_gb300.studies convergence --kind cdft --max-n 256 --out results/...
    python -m paper_1503_07416_gb300.studies freezing --kind cdft --steps 50000 --every 100 --out results/...
"""
from __future__ import annotations

import argparse
import json
import math
import os
import time

import numpy as np

from . import fm, inputs

# The paper's Cauchy errors ||e^{h;h/2}|| for the pairs 16-32, 32-64, 64-128,
# 128-256, 256-512 (Tables 1-3: CDFT rho, u, v; Tables 4-6: PFC rho, u, v).
PAPER_TABLES = {
    ("cdft", "rho"): [4.4800e-5, 2.4951e-7, 4.8685e-8, 1.0802e-8, 2.2465e-9],
    ("cdft", "u"): [5.3251e-5, 2.4077e-7, 4.6670e-8, 1.0715e-8, 2.5396e-9],
    ("cdft", "v"): [5.3467e-5, 2.5007e-7, 4.8696e-8, 1.1342e-8, 2.7102e-9],
    ("pfc", "rho"): [5.9041e-6, 1.1318e-6, 2.6468e-7, 6.2968e-8, 1.5300e-8],
    ("pfc", "u"): [7.8360e-7, 1.3122e-7, 2.5793e-8, 5.6521e-9, 1.3191e-9],
    ("pfc", "v"): [6.6965e-7, 1.4285e-7, 3.2625e-8, 7.7450e-9, 1.8833e-9],
}

L_CONV = 32.0       # Sec. 6.1: [0, 32)^2
T_FINAL = 10.0      # t_f
CDFT_NU_CONV = 1.0  # Sec. 6.1.1: nu = 1
PFC_ALPHA_CONV = 0.975  # Sec. 6.1.2: eps = 0.025


def _solver(kind, n, h, precision, tol, stream=None, **kw):
    extra = dict(alpha=PFC_ALPHA_CONV) if kind == "pfc" else dict(nu=CDFT_NU_CONV, delta=1e-10)
    extra.update(kw)
    return fm.Solver(kind, (n, n), h, precision=precision, tol=tol, max_cycles=200, stream=stream, **extra)


def evolve(kind, n, t_final=T_FINAL, tol=1e-12, precision=fm.FM_FP64, w_damp=0.0, pfc_offset=1.5):
    """Evolve the smooth convergence-test field on an n^2 grid to t_final
    along s = 0.025 h^2.  Returns (rho, [u, v], info dict).  The tolerance is
    raised by decades (up to 1e-9) if the first step cannot reach it (the
    round-off floor of the weighted residual grows as h falls)."""
    import torch
    rho0, h = inputs.smooth_convergence_field(n, L=L_CONV, kind=kind, pfc_offset=pfc_offset)
    s = 0.025 * h * h
    nsteps = int(round(t_final / s))
    vel0 = [np.zeros_like(rho0), np.zeros_like(rho0)]
    stream = torch.cuda.current_stream().cuda_stream
    while True:
        sol = _solver(kind, n, h, precision, tol, stream=stream, w_damp=w_damp)
        rho_d = torch.from_numpy(rho0).cuda()
        vel_d = [torch.from_numpy(v).cuda() for v in vel0]
        sol.set_fields(rho_d, vel_d)
        code, info = fm.fm_step_raw(sol.handle, s)
        if code == fm.FM_ENOCONV and tol < 1e-9:
            sol.close()
            tol *= 10.0
            continue
        if code != fm.FM_OK:
            raise fm.FMError(code, f"step 1 of the {n}^2 {kind} convergence run")
        break
    cycles = [info.cycles]
    t0 = time.perf_counter()
    for k in range(1, nsteps):
        info = sol.step(s)
        cycles.append(info.cycles)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    rho, vel = sol.get_fields()
    sol.close()
    return rho, vel, dict(n=n, h=h, s=s, steps=nsteps, tol=tol, cycles_mean=float(np.mean(cycles)),
                          cycles_max=int(max(cycles)), wall_s=wall)


def cauchy_errors(coarse, fine, h_coarse):
    """||e^{h;h/2}||_2 = sqrt(h^2 sum (f^h_{ij} - f^{h/2}_{2i,2j})^2) with the
    coarse spacing h."""
    e = coarse - fine[::2, ::2]
    return math.sqrt(h_coarse * h_coarse * float(np.sum(e * e)))


def convergence(kind, sizes=(16, 32, 64, 128, 256), t_final=T_FINAL, tol=1e-12, pfc_offset=1.5):
    """Run the refinement study; returns a dict with the per-grid runs, the
    Cauchy errors and rates of rho, u, v, and the paper's values beside them."""
    sols = {}
    runs = []
    for n in sizes:
        rho, vel, info = evolve(kind, n, t_final=t_final, tol=tol, pfc_offset=pfc_offset)
        sols[n] = (rho, vel[0], vel[1], info["h"])
        runs.append(info)
    fields = ["rho", "u", "v"]
    errs = {f: [] for f in fields}
    pairs = []
    for a, b in zip(sizes[:-1], sizes[1:]):
        pairs.append(f"{a}-{b}")
        for k, f in enumerate(fields):
            errs[f].append(cauchy_errors(sols[a][k], sols[b][k], sols[a][3]))
    rates = {f: [None] + [math.log2(x / y) if y > 0 else None for x, y in zip(v[:-1], v[1:])]
             for f, v in errs.items()}
    paper = {}
    for f in fields:
        tab = PAPER_TABLES[(kind, f)]
        idx = [int(math.log2(a // 16)) for a in sizes[:-1]]
        paper[f] = [tab[i] if 0 <= i < len(tab) else None for i in idx]
    return dict(kind=kind, t_final=t_final, sizes=list(sizes), pairs=pairs, runs=runs, errors=errs,
                rates=rates, paper=paper, pfc_offset=pfc_offset if kind == "pfc" else None)


def convergence_markdown(res):
    """The study as a markdown table, ours beside the paper's."""
    kind = res["kind"]
    tabs = {"cdft": "Tables 1-3", "pfc": "Tables 4-6"}[kind]
    lines = [f"# Convergence study, {kind.upper()} (Sec. 6.1, {tabs})", "",
             f"Smooth initial density of Sec. 6.1 on [0, 32)^2"
             + (f" (PFC offset {res['pfc_offset']})" if res.get("pfc_offset") is not None else "")
             + f", u = 0, t_f = {res['t_final']}, "
             "s = 0.025 h^2, float64 path of libfm on one GB300.  ||e|| = sqrt(h^2 sum e^2) with the "
             "coarse spacing; rate = log2 of consecutive error ratios.", "",
             "| pair | field | ||e|| (ours) | rate (ours) | ||e|| (paper) | rate (paper) |",
             "|---|---|---|---|---|---|"]
    for f in ("rho", "u", "v"):
        pap = res["paper"][f]
        for k, pair in enumerate(res["pairs"]):
            ours = res["errors"][f][k]
            r = res["rates"][f][k]
            pr = None
            if k > 0 and pap[k] and pap[k - 1]:
                pr = math.log2(pap[k - 1] / pap[k])
            lines.append(f"| {pair} | {f} | {ours:.4e} | {'' if r is None else f'{r:.2f}'} | "
                         f"{'' if pap[k] is None else f'{pap[k]:.4e}'} | {'' if pr is None else f'{pr:.2f}'} |")
    lines += ["", "| grid | h | s | steps | tol | V-cycles per step (mean / max) | wall s |",
              "|---|---|---|---|---|---|---|"]
    for r in res["runs"]:
        lines.append(f"| {r['n']}^2 | {r['h']:.4g} | {r['s']:.4g} | {r['steps']} | {r['tol']:.0e} | "
                     f"{r['cycles_mean']:.2f} / {r['cycles_max']} | {r['wall_s']:.1f} |")
    return "\n".join(lines) + "\n"


def freezing(kind, steps, every=100, n=128, precision=fm.FM_MIXED, tol=1e-10, w_damp=0.5, seed=11, out=None,
             nu=2.362, coarsest=16, ncoarse=4):
    """Freeze a supercooled liquid for `steps` steps; returns the list of
    logged records (every `every` steps and the first and last) and a
    summary.  E is evaluated at every step and must not increase (beyond
    1e-12 relative, the solver tolerance's effect)."""
    import torch
    rho, vel, prm = inputs.freezing(kind, n, seed, nu=nu)
    h, dt = prm["h"], prm["dt"]
    extra = dict(nu=prm["nu"], delta=prm["delta"]) if kind == "cdft" else dict(alpha=prm["alpha"])
    stream = torch.cuda.current_stream().cuda_stream
    sol = fm.Solver(kind, (n, n), h, precision=precision, tol=tol, w_damp=w_damp, max_cycles=200,
                    coarsest=coarsest, ncoarse=ncoarse, stream=stream, **extra)
    sol.set_fields(rho, vel)
    M0 = sol.mass()
    recs = []
    E_prev = None
    worst_rise = 0.0
    t0 = time.perf_counter()
    fh = open(out, "w") if out else None
    for k in range(steps + 1):
        info = None
        if k > 0:
            code, info = fm.fm_step_raw(sol.handle, dt)
            if code != fm.FM_OK:  # record where the solve stopped and end the run
                rec = dict(step=k, t=round(k * dt, 10), failed=fm.strerror(code), cycles=info.cycles, res=info.res)
                recs.append(rec)
                if fh:
                    fh.write(json.dumps(rec) + "\n")
                steps = k - 1
                break
        terms = sol.energy_terms()
        KE = terms[0]
        F = sum(terms[1:])
        E = KE + F
        if E_prev is not None:
            worst_rise = max(worst_rise, (E - E_prev) / max(1.0, abs(E_prev)))
        E_prev = E
        if k % every == 0 or k == steps:
            rec = dict(step=k, t=round(k * dt, 10), E=E, F=F, KE=KE, mass=sol.mass(),
                       cycles=info.cycles if info else 0, res=info.res if info else None,
                       wall_s=round(time.perf_counter() - t0, 3))
            if kind == "cdft":
                rec.update(F_id=terms[1], F_ex=terms[2])
            else:
                rec.update(F_quartic=terms[1], F_quadratic=terms[2], F_lap2=terms[3], F_rho_lap=terms[4])
            recs.append(rec)
            if fh:
                fh.write(json.dumps(rec) + "\n")
    if fh:
        fh.close()
    sol.close()
    good = [r for r in recs if "failed" not in r]
    summary = dict(kind=kind, n=n, h=h, dt=dt, nu=prm.get("nu"), steps=steps, precision="mixed" if precision else "fp64",
                   coarsest=coarsest, ncoarse=ncoarse, stopped=recs[-1].get("failed"),
                   tol=tol, w_damp=w_damp, energy_max_relative_rise=worst_rise,
                   mass_drift=abs(good[-1]["mass"] - M0) / abs(M0), KE_peak_t=max(good, key=lambda r: r["KE"])["t"],
                   wall_s=good[-1]["wall_s"])
    if kind == "cdft":
        summary.update(F_id_change=good[-1]["F_id"] - good[0]["F_id"], F_ex_change=good[-1]["F_ex"] - good[0]["F_ex"])
    return recs, summary


def shear(n=256, anneal=2000, drive=2000, u_wall=0.1, every=50, precision=fm.FM_MIXED, tol=1e-10, out=None):
    """Sec. 6.3: the hexagonal nanocrystal in its liquid between walls,
    annealed with the walls at rest for `anneal` steps (the energy must not
    increase: Thm 5.1 with no-slip walls at rest), then driven with the walls
    at -u_wall (bottom) and +u_wall (top) for `drive` steps (a driven system:
    the energy may rise).  Returns the logged records and a summary."""
    import torch
    rho, vel, prm = inputs.nanocrystal(n)
    stream = torch.cuda.current_stream().cuda_stream
    recs = []
    fh = open(out, "w") if out else None
    t0 = time.perf_counter()
    worst_rise = 0.0
    k = 0
    for phase, nsteps, walls in (("anneal", anneal, (0.0, 0.0)), ("drive", drive, (-u_wall, u_wall))):
        sol = fm.Solver("pfc", (n, n), prm["h"], alpha=prm["alpha"], precision=precision, tol=tol, w_damp=0.0,
                        max_cycles=200, walls=fm.FM_WALLS_Y, u_wall=walls, stream=stream)
        sol.set_fields(rho, vel)
        E_prev = None
        for j in range(nsteps + 1):
            info = sol.step(prm["dt"]) if j > 0 else None
            if j > 0:
                k += 1
            if j % every == 0 or j == nsteps:
                E, F, KE = sol.energy()
                if phase == "anneal" and E_prev is not None:
                    worst_rise = max(worst_rise, (E - E_prev) / max(1.0, abs(E_prev)))
                E_prev = E if phase == "anneal" else None
                rec = dict(phase=phase, step=k, t=round(k * prm["dt"], 10), E=E, F=F, KE=KE, mass=sol.mass(),
                           cycles=info.cycles if info else 0, wall_s=round(time.perf_counter() - t0, 3))
                recs.append(rec)
                if fh:
                    fh.write(json.dumps(rec) + "\n")
        rho, vel = sol.get_fields()
        sol.close()
    if fh:
        fh.close()
    an = [r for r in recs if r["phase"] == "anneal"]
    dr = [r for r in recs if r["phase"] == "drive"]
    summary = dict(n=n, h=prm["h"], dt=prm["dt"], anneal_steps=anneal, drive_steps=drive, u_wall=u_wall,
                   anneal_energy_max_relative_rise_between_logs=worst_rise,
                   anneal_E=(an[0]["E"], an[-1]["E"]), drive_E=(dr[0]["E"], dr[-1]["E"]),
                   drive_KE=(dr[0]["KE"], dr[-1]["KE"]), mass_drift=abs(recs[-1]["mass"] - recs[0]["mass"]) / recs[0]["mass"],
                   wall_s=recs[-1]["wall_s"])
    return recs, summary


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    sub = ap.add_subparsers(dest="cmd", required=True)
    c = sub.add_parser("convergence")
    c.add_argument("--kind", choices=["cdft", "pfc"], required=True)
    c.add_argument("--max-n", type=int, default=256)
    c.add_argument("--t-final", type=float, default=T_FINAL)
    c.add_argument("--pfc-offset", type=float, default=1.5)
    c.add_argument("--out", default=None)
    f = sub.add_parser("freezing")
    f.add_argument("--kind", choices=["cdft", "pfc"], required=True)
    f.add_argument("--steps", type=int, default=50000)
    f.add_argument("--every", type=int, default=100)
    f.add_argument("--out", default=None, help="JSONL log of the records")
    f.add_argument("--summary", default=None)
    f.add_argument("--nu", type=float, default=2.362)
    f.add_argument("--coarsest", type=int, default=16)
    f.add_argument("--ncoarse", type=int, default=4)
    sh = sub.add_parser("shear")
    sh.add_argument("--n", type=int, default=256)
    sh.add_argument("--anneal", type=int, default=2000)
    sh.add_argument("--drive", type=int, default=2000)
    sh.add_argument("--u-wall", type=float, default=0.1)
    sh.add_argument("--every", type=int, default=50)
    sh.add_argument("--out", default=None)
    sh.add_argument("--summary", default=None)
    args = ap.parse_args()
    import torch
    torch.cuda.set_device(0)
    from . import build
    build.build_library()
    if args.cmd == "convergence":
        sizes = tuple(16 << k for k in range(int(math.log2(args.max_n // 16)) + 1))
        res = convergence(args.kind, sizes, t_final=args.t_final, pfc_offset=args.pfc_offset)
        md = convergence_markdown(res)
        print(md)
        if args.out:
            os.makedirs(os.path.dirname(os.path.abspath(args.out)), exist_ok=True)
            with open(args.out, "w") as fh:
                fh.write(md)
            with open(os.path.splitext(args.out)[0] + ".json", "w") as fh:
                json.dump(res, fh, indent=1)
    else:
        if args.cmd == "freezing":
            recs, summary = freezing(args.kind, args.steps, args.every, out=args.out, nu=args.nu,
                                     coarsest=args.coarsest, ncoarse=args.ncoarse)
        else:
            recs, summary = shear(args.n, args.anneal, args.drive, args.u_wall, args.every, out=args.out)
        print(json.dumps(summary))
        if args.summary:
            with open(args.summary, "w") as fh:
                json.dump(summary, fh, indent=1)


if __name__ == "__main__":
    main()
