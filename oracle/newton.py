"""Dense Newton solve of N(g) = S on tiny grids (brute force).

TEST INFRASTRUCTURE ONLY (see ``oracle/scheme.py``).

The Jacobian is assembled column by column with the complex step
dN/dg_j = Im N(g + i t e_j) / t, which is exact to rounding for the analytic
operator N of App. G; each Newton correction is a dense LU solve (numpy).
It solves the same discrete scheme as the FAS solver without any multigrid or
smoothing, so the two can be checked against each other.
"""
from __future__ import annotations

import math

import numpy as np

from . import scheme


def _pack(g):
    return np.concatenate([x.ravel() for x in g])


def _unpack(x, shape, k):
    n = int(np.prod(shape))
    return [x[i * n:(i + 1) * n].reshape(shape) for i in range(k)]


def solve_dense(rho, vel, P: scheme.Params, J=None, tol=1e-13, max_iter=30):
    """One time step with N(g) = S solved by dense Newton.

    Returns (rho^{k+1} after the closure, velocity, g, residual norm)."""
    om = scheme.vorticity(vel, P.h)
    C = scheme.conv_fft(J, rho, P.h) if P.kind == scheme.CDFT else None
    S = scheme.source(rho, vel, om, P, C)
    c = scheme.Coeffs(rho, om)
    g = scheme.initial_iterate(rho, vel, P)
    shape = rho.shape
    k = len(g)
    x = _pack(g)
    Sv = _pack(S)
    t = 1e-30
    nr = math.inf
    for _ in range(max_iter):
        gx = _unpack(x, shape, k)
        F = _pack(scheme.apply_N(gx, c, P)) - Sv
        nr = scheme.res_norm(_unpack(F, shape, k), P.h)
        if nr <= tol:
            break
        m = x.size
        Jm = np.empty((m, m))
        for j in range(m):
            xc = x.astype(complex)
            xc[j] += 1j * t
            Jm[:, j] = np.imag(_pack(scheme.apply_N(_unpack(xc, shape, k), c, P))) / t
        x = x - np.linalg.solve(Jm, F)
    g = _unpack(x, shape, k)
    rho_new = scheme.closure(g, rho, vel, P)
    return rho_new, [y.copy() for y in g[1:1 + P.dim]], g, nr
