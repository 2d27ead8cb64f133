"""Seeded synthetic initial states and the parameter sets of the workloads.

This module holds no arithmetic of the numerical method: it only draws seeded
initial fields (noise, Gaussian nuclei, the smooth convergence-test fields of
Sec. 6.1) and names the physical parameters of each workload.  Both the CUDA
path's tests and benchmarks and the CPU oracle's tests use it.

Workloads (all periodic, gamma = 2, V(2,2) cycles):

* ``pfc64``     2-D PFC 64x64, L = 32 (h = 0.5), eps = 0.025 (alpha = 0.975),
                rho = 3/2 - 0.07 sqrt(3) + 0.01 U(-1,1), u = 0, s = 0.01,
                10 steps, tol 1e-10, w_damp 0.5, delta 0 (Sec. 6.2 PFC freezing).
* ``pfc512``    2-D PFC 512x512, h = pi/(2 sqrt 3) (Sec. 6.3), eps = 0.4
                (alpha = 0.6), supercooled liquid rho = 0.80 plus four seeded
                Gaussian nuclei (amplitude 0.5, width a/2, a = 4 pi/sqrt 3)
                plus 0.01 U(-1,1), s = 0.02, 200 steps, tol 1e-10.
* ``cdft256``   2-D CDFT 256x256, h = 17/128 (L = 34), nu = 2.362,
                rho = 0.1 pi (1 + 0.1 eta), eta ~ U[0,1], s = 0.02,
                delta = 1e-10, 100 steps (Sec. 6.2 CDFT freezing).
* ``batch48``   48 independent 2-D PFC instances with the ``pfc512`` physics,
                n drawn from {128, 256, 512, 1024}, dt log-uniform in
                [1e-3, 1e-1], 20 steps each.
* ``pfc3d128``  3-D PFC 128^3, h = pi/(2 sqrt 3), eps = 0.4, rho = 0.80 +
                0.01 U(-1,1) plus one spherical Gaussian nucleus, s = 0.02,
                50 steps.
"""
from __future__ import annotations

import math

import numpy as np

H_HEX = math.pi / (2.0 * math.sqrt(3.0))     # Sec. 6.3 grid spacing
A_ATOM = 4.0 * math.pi / math.sqrt(3.0)      # Sec. 6.3 atom size


# Multigrid depth the large 2-D workloads (pfc512, cdft256, batch48) are
# timed with: coarsen down to 64 points per side, two sweeps on the coarsest
# grid (the library defaults are 16 and 4).  At these time steps the cycle
# counts of these workloads are the same either way; the shallower
# hierarchy saves latency-bound coarse-level launches.
BENCH_MG_2D = dict(coarsest=64, ncoarse=2)


def uniform_noise(shape, seed, lo=-1.0, hi=1.0):
    return np.random.default_rng(seed).uniform(lo, hi, size=shape)


def gaussian_nuclei(shape, h, centres, amp, width):
    """Sum of periodic Gaussian bumps amp * exp(-|x - c|^2 / (2 width^2))
    (minimum-image distance)."""
    nd = len(shape)
    out = np.zeros(shape)
    L = [n * h for n in shape]
    axes = []
    for ax in range(nd):
        n = shape[ax]
        axes.append(np.arange(n) * h)
    for c in centres:
        r2 = np.zeros(shape)
        for ax in range(nd):
            dx = np.abs(axes[ax] - c[ax])
            dx = np.minimum(dx, L[ax] - dx)
            bshape = [1] * nd
            bshape[ax] = shape[ax]
            r2 = r2 + (dx ** 2).reshape(bshape)
        out += amp * np.exp(-r2 / (2.0 * width * width))
    return out


def pfc64(seed=1, n=64):
    """Returns (rho, vel, params dict).  Array axes are [y][x]."""
    h = 32.0 / n
    rho = (1.5 - 0.07 * math.sqrt(3.0)) + 0.01 * uniform_noise((n, n), seed)
    vel = [np.zeros((n, n)), np.zeros((n, n))]
    prm = dict(kind="pfc", dim=2, n=n, h=h, dt=0.01, alpha=0.975, gamma=2.0,
               delta=0.0, w_damp=0.5, tol=1e-10, steps=10)
    return rho, vel, prm


def pfc_supercooled(n, seed, dim=2, nuclei=4, rho_bar=0.80, dt=0.02):
    h = H_HEX
    shape = (n,) * dim
    rng = np.random.default_rng(seed)
    L = n * h
    centres = rng.uniform(0.0, L, size=(nuclei, dim))
    rho = rho_bar + gaussian_nuclei(shape, h, centres[:, ::-1], 0.5, A_ATOM / 2.0)
    rho = rho + 0.01 * rng.uniform(-1.0, 1.0, size=shape)
    vel = [np.zeros(shape) for _ in range(dim)]
    prm = dict(kind="pfc", dim=dim, n=n, h=h, dt=dt, alpha=0.6, gamma=2.0,
               delta=0.0, w_damp=0.5, tol=1e-10)
    return rho, vel, prm


def pfc512(seed=2, n=512):
    rho, vel, prm = pfc_supercooled(n, seed)
    prm["steps"] = 200
    return rho, vel, prm


def cdft256(seed=3, n=256):
    h = 34.0 / n
    rho_bar = 0.1 * math.pi
    eta = np.random.default_rng(seed).uniform(0.0, 1.0, size=(n, n))
    rho = rho_bar * (1.0 + 0.1 * eta)
    vel = [np.zeros((n, n)), np.zeros((n, n))]
    prm = dict(kind="cdft", dim=2, n=n, h=h, dt=0.02, nu=2.362, gamma=2.0,
               delta=1e-10, w_damp=0.5, tol=1e-10, steps=100)
    return rho, vel, prm


def batch48(seed=4, count=48, sizes=(128, 256, 512, 1024)):
    """List of (rho, vel, params) for independent instances."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(rng.choice(sizes))
        dt = float(math.exp(rng.uniform(math.log(1e-3), math.log(1e-1))))
        rho, vel, prm = pfc_supercooled(n, seed * 1000 + i, dt=dt)
        prm["steps"] = 20
        out.append((rho, vel, prm))
    return out


def pfc3d128(seed=5, n=128):
    h = H_HEX
    L = n * h
    shape = (n, n, n)
    rng = np.random.default_rng(seed)
    rho = 0.80 + 0.01 * rng.uniform(-1.0, 1.0, size=shape)
    rho = rho + gaussian_nuclei(shape, h, [(L / 2, L / 2, L / 2)], 0.5, A_ATOM / 2.0)
    vel = [np.zeros(shape) for _ in range(3)]
    prm = dict(kind="pfc", dim=3, n=n, h=h, dt=0.02, alpha=0.6, gamma=2.0,
               delta=0.0, w_damp=0.5, tol=1e-10, steps=50)
    return rho, vel, prm


def freezing(kind, n=128, seed=11, nu=2.362):
    """Sec. 6.2 freezing runs: rho = rho_bar (1 + 0.1 eta), eta ~ U[0, 1],
    u = 0.  CDFT: rho_bar = 0.1 pi (packing fraction 0.6), [0, 17)^2,
    nu = 2.362, s = 0.02, delta = 1e-10.  PFC: rho_bar = 3/2 - 0.07 sqrt 3
    (the 3/2 offset of the psi <-> rho map, see the design notes),
    [0, 32)^2, eps = 0.025 (alpha = 0.975), s = 0.01."""
    eta = np.random.default_rng(seed).uniform(0.0, 1.0, size=(n, n))
    vel = [np.zeros((n, n)), np.zeros((n, n))]
    if kind == "cdft":
        rb, L = 0.1 * math.pi, 17.0
        prm = dict(kind="cdft", dim=2, n=n, h=L / n, dt=0.02, nu=nu, gamma=2.0, delta=1e-10)
    else:
        rb, L = 1.5 - 0.07 * math.sqrt(3.0), 32.0
        prm = dict(kind="pfc", dim=2, n=n, h=L / n, dt=0.01, alpha=0.975, gamma=2.0, delta=0.0)
    return rb * (1.0 + 0.1 * eta), vel, prm


def nanocrystal(n=256, eps=0.4, rho_s=0.90073, rho_l=0.72958, diag_atoms=13.0):
    """Sec. 6.3 channel test: an n x n grid with h = pi/(2 sqrt 3) (L = n h),
    liquid rho_l everywhere except a regular hexagon of long diagonal
    13 a centred at (L/2, L/2), a = 4 pi / sqrt 3, filled with the one-mode
    solid rho_s + A (cos(sqrt(3)/2 x + pi) cos(y/2) - cos(y)/2) with the
    amplitude A printed in Sec. 6.3 (A = 4/(5 sqrt 3) (rho_s - 3/2)
    - (4 sqrt 3 / 15) sqrt(15 eps - 12 (rho_s - 3/2)^2)); u = 0.  y is measured
    at the cell centres (j + 1/2) h between the walls."""
    h = H_HEX
    L = n * h
    x = np.arange(n) * h
    y = (np.arange(n) + 0.5) * h
    X, Y = np.meshgrid(x, y, indexing="xy")
    d = rho_s - 1.5
    A = 4.0 / (5.0 * math.sqrt(3.0)) * d - 4.0 * math.sqrt(3.0) / 15.0 * math.sqrt(15.0 * eps - 12.0 * d * d)
    solid = rho_s + A * (np.cos(math.sqrt(3.0) / 2.0 * X + math.pi) * np.cos(Y / 2.0) - 0.5 * np.cos(Y))
    R = 0.5 * diag_atoms * A_ATOM              # circumradius of the hexagon
    px, py = np.abs(X - L / 2), np.abs(Y - L / 2)
    inside = (py <= R * math.sqrt(3.0) / 2.0) & (math.sqrt(3.0) * px + py <= math.sqrt(3.0) * R)
    rho = np.where(inside, solid, rho_l)
    vel = [np.zeros((n, n)), np.zeros((n, n))]
    prm = dict(kind="pfc", dim=2, n=n, h=h, dt=0.02, alpha=1.0 - eps, gamma=2.0, delta=0.0)
    return rho, vel, prm


def smooth_convergence_field(n, L=32.0, kind="pfc", pfc_offset=1.5):
    """The smooth initial density of the convergence tests (Sec. 6.1.1 CDFT,
    Sec. 6.1.2 PFC; for PFC the offset 3/2 of the psi <-> rho map is used by
    default, pfc_offset = 0.5 gives the text's literal value, see the design
    notes)."""
    h = L / n
    x = np.arange(n) * h
    X, Y = np.meshgrid(x, x, indexing="xy")
    pert = (-0.02 * np.cos(2 * math.pi * (X - 12.0) / 32.0) * np.sin(2 * math.pi * (Y - 1.0) / 32.0)
            + 0.02 * np.cos(math.pi * (X + 10.0) / 32.0) ** 2 * np.cos(math.pi * (Y + 3.0) / 32.0) ** 2
            - 0.01 * np.sin(4 * math.pi * X / 32.0) ** 2 * np.sin(4 * math.pi * (Y - 6.0) / 32.0) ** 2)
    if kind == "pfc":
        return math.sqrt(3.0) * (-0.07 + pert) + pfc_offset, h
    return math.pi / 6.0 * 0.6 + pert, h
