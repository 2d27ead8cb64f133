"""Plain FP64 CPU oracle of the conservative gradient-flow scheme.

TEST INFRASTRUCTURE ONLY, under the same rule as ``oracle.scheme``: only
``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU legs import it;
the product path never does.

What is computed (Sec. 3, Thm 3.3, Eq. gradient_scheme): one implicit step of

    rho^{k+1} - rho^k = s Lap_h ( dF_c[rho^{k+1}] - dF_e[rho^k] ),

with the discrete functionals and convex splittings of Sec. 5.2 (CDFT, Lemma
5.2) and Sec. 5.3 (PFC, Lemma 5.4) and the operators of App. E (periodic),
solved by the same FAS multigrid as the hydrodynamic step (``oracle.scheme``:
nodal full weighting, injection, bilinear prolongation, red-black point
Gauss-Seidel with damping, reading R6).

Unknowns per point (readings, see below):
  PFC  g = (rho, mu, kappa):  N1 = rho - s Lap_h mu            = rho^k
                              N2 = mu - psi^3/3 - alpha psi - Lap_h kappa
                                                              = 2 Lap_h rho^k
                              N3 = kappa - Lap_h rho           = 0
  CDFT g = (rho,):            N1 = rho - s Lap_h (ln rho + 2 c_e rho)
                                 = rho^k - s Lap_h (2 c_e rho^k + J * rho^k)

Readings (the paper states the scheme, not its discretisation or solver):
GF1 Lap_h is the 5-point (7-point in 3-D) Laplacian of App. E, so the scheme
    conserves (rho || 1) exactly and the energy argument of Thm 3.3 goes
    through with the edge norms: F^{k+1} - F^k <= -s h^d sum_edges |D mu|^2.
GF2 PFC carries mu and kappa = Lap_h rho as unknowns, as the hydrodynamic
    PFC system of App. G.2 does; CDFT eliminates mu (it is a function of
    the point's own rho).
GF3 Point block: PFC solves the 3x3 system of (rho, mu, kappa) at the point
    with the cubic linearised about the current rho (as App. G.2 does);
    CDFT takes one Newton step on its scalar point equation about the
    current rho.  Then the projection and the damping of ``oracle.scheme``
    (readings R7, R8).
GF4 Closure (as reading R10): after the solve rho^{k+1} is re-evaluated as
    rho^k + s Lap_h mu with the converged mu, so mass is exact to round-off,
    then projected.
GF5 Initial iterate: rho^k; PFC kappa^0 = Lap_h rho^k and mu^0 the N2 value
    at rho^k (as reading R11).
"""
from __future__ import annotations

import math

import numpy as np

from . import scheme as S


def nunk(P):
    return 3 if P.kind == S.PFC else 1


def explicit_mu(rk, P, C=None):
    """-dF_e[rho^k]: 2 Lap_h rho^k (PFC, Lemma 5.4) or -(2 c_e rho^k + J * rho^k)
    (CDFT, Lemma 5.2)."""
    if P.kind == S.PFC:
        return 2.0 * S.lap(rk, P.h)
    return -(2.0 * P.ce * rk + C)


def mu_of(g, P, Emu=None):
    """mu^{k+1} = dF_c[rho] - dF_e[rho^k] of an iterate: the unknown mu (PFC)
    or ln rho + 2 c_e rho + Emu (CDFT, Emu = explicit_mu)."""
    if P.kind == S.PFC:
        return g[1]
    return np.log(g[0]) + 2.0 * P.ce * g[0] + (0.0 if Emu is None else Emu)


def apply_N(g, P):
    """N(g) (the implicit parts; CDFT's explicit potential enters S)."""
    h, s = P.h, P.s
    if P.kind == S.PFC:
        rho, mu, kap = g
        psi = rho - 1.5
        return [rho - s * S.lap(mu, h),
                mu - psi ** 3 / 3.0 - P.alpha * psi - S.lap(kap, h),
                kap - S.lap(rho, h)]
    rho = g[0]
    return [rho - s * S.lap(np.log(rho) + 2.0 * P.ce * rho, h)]


def source(rk, P, C=None):
    """S: rho^k and the explicit potential (PFC: S2 = 2 Lap_h rho^k; CDFT:
    S1 = rho^k + s Lap_h (-(2 c_e rho^k + J * rho^k)))."""
    if P.kind == S.PFC:
        return [rk.copy(), explicit_mu(rk, P), np.zeros_like(rk)]
    return [rk + P.s * S.lap(explicit_mu(rk, P, C), P.h)]


def residual(g, f, P):
    N = apply_N(g, P)
    return [f[i] - N[i] for i in range(len(f))]


def point_update(g, f, P, mask):
    """Point block at the points of ``mask`` (no two are neighbours), all
    other points fixed (reading GF3), then projection and damping."""
    h, s, d = P.h, P.s, g[0].ndim
    old = [x.copy() for x in g]
    w = P.w_damp
    c = 2.0 * d / (h * h)
    if P.kind == S.PFC:
        rho, mu, kap = g
        a = s * c
        b1 = f[0] + s * S.nb_sum(mu) / (h * h)
        b3 = f[2] + S.nb_sum(rho) / (h * h)
        psl = rho - 1.5
        q = psl * psl + P.alpha
        # cubic linearised about the current rho: psi^3/3 ~ psl^2 psi - 2 psl^3/3
        b2 = f[1] + S.nb_sum(kap) / (h * h) - (2.0 / 3.0) * psl ** 3 - 1.5 * q
        # rho + a mu = b1;  mu - q rho + c kappa = b2;  kappa + c rho = b3
        mu_new = (b2 + (q + c * c) * b1 - c * b3) / (1.0 + a * (q + c * c))
        rho_new = b1 - a * mu_new
        rho_new = np.sqrt(rho_new * rho_new + P.delta * P.delta)
        kap_new = b3 - c * rho_new
        new = [rho_new, mu_new, kap_new]
    else:
        rho = g[0]
        a = s * c
        m_nb = S.nb_sum(np.log(rho) + 2.0 * P.ce * rho) / (h * h)
        b = f[0] + s * m_nb
        # one Newton step on rho + a (ln rho + 2 c_e rho) = b about the current rho
        F = rho + a * (np.log(rho) + 2.0 * P.ce * rho) - b
        dF = 1.0 + a * (1.0 / rho + 2.0 * P.ce)
        rho_new = rho - F / dF
        new = [np.sqrt(rho_new * rho_new + P.delta * P.delta)]
    for i in range(len(g)):
        g[i] = np.where(mask, (1.0 - w) * new[i] + w * old[i], g[i])


def smooth(g, f, P, ordering="redblack"):
    if ordering == "redblack":
        for m in S.color_masks(g[0].shape):
            point_update(g, f, P, m)
    else:
        shape = g[0].shape
        for p in np.ndindex(*shape):
            m = np.zeros(shape, dtype=bool)
            m[p] = True
            point_update(g, f, P, m)


def vcycle(g, f, P, opts):
    """FAS V(nu1, nu2) cycle on N(g) = f (as ``scheme.vcycle``)."""
    if not S.can_coarsen(g[0].shape, opts):
        for _ in range(opts.ncoarse):
            smooth(g, f, P, opts.ordering)
        return
    for _ in range(opts.nu1):
        smooth(g, f, P, opts.ordering)
    r = residual(g, f, P)
    PH = P.coarse()
    gH = [S.inject(x) for x in g]
    NH = apply_N(gH, PH)
    fH = [NH[i] + S.restrict_fw(r[i]) for i in range(len(r))]
    gH0 = [x.copy() for x in gH]
    vcycle(gH, fH, PH, opts)
    for i in range(len(g)):
        g[i] = g[i] + S.prolong(gH[i] - gH0[i])
    if P.delta > 0.0:
        g[0] = np.sqrt(g[0] * g[0] + P.delta * P.delta)  # reading R8
    for _ in range(opts.nu2):
        smooth(g, f, P, opts.ordering)


def initial_iterate(rk, P):
    """Reading GF5."""
    if P.kind == S.PFC:
        kap0 = S.lap(rk, P.h)
        psi = rk - 1.5
        mu0 = psi ** 3 / 3.0 + P.alpha * psi + S.lap(kap0, P.h) + 2.0 * S.lap(rk, P.h)
        return [rk.copy(), mu0, kap0]
    return [rk.copy()]


def closure(g, rk, P, Emu=None):
    """Reading GF4: rho^{k+1} = rho^k + s Lap_h mu^{k+1}, projected."""
    rho = rk + P.s * S.lap(mu_of(g, P, Emu), P.h)
    return np.sqrt(rho * rho + P.delta * P.delta)


def step(rho, P, opts=None, J=None):
    """One gradient-flow step of size P.s.  Returns (rho^{k+1}, info) with
    info: cycles, residual history, converged iterate g, source S, mu^{k+1}."""
    opts = opts or S.SolverOpts()
    C = S.conv_fft(J, rho, P.h) if P.kind == S.CDFT else None
    f = source(rho, P, C)
    Emu = explicit_mu(rho, P, C) if P.kind == S.CDFT else None
    g = initial_iterate(rho, P)
    hist, cycles = [], 0
    while True:
        nr = S.res_norm(residual(g, f, P), P.h)
        hist.append(nr)
        if not math.isfinite(nr):
            raise S.NoConvergence("non-finite residual")
        if nr <= opts.tol:
            break
        if cycles >= opts.max_cycles:
            raise S.NoConvergence(f"no convergence after {cycles} cycles: {hist}")
        vcycle(g, f, P, opts)
        cycles += 1
    mu = mu_of(g, P, Emu)
    return closure(g, rho, P, Emu), dict(cycles=cycles, hist=hist, g=g, S=f, mu=mu)


def free_energy(rho, P, J=None):
    return S.free_energy(rho, P, J)


def edge_norm(a, h):
    """h^d sum over edges of (D_d a)^2, the discrete ||grad a||^2."""
    acc = 0.0
    for d in range(a.ndim):
        Dd = (S.sh(a, d, 1) - a) / h
        acc += float(np.sum(Dd * Dd)) * h ** a.ndim
    return acc


def solve_dense(rho, P, J=None, tol=1e-13, max_iter=60):
    """N(g) = S by dense Newton (complex-step Jacobian) on a tiny grid, with no
    multigrid involved.  Returns (rho^{k+1}, g, residual norm)."""
    C = S.conv_fft(J, rho, P.h) if P.kind == S.CDFT else None
    f = source(rho, P, C)
    Emu = explicit_mu(rho, P, C) if P.kind == S.CDFT else None
    g = initial_iterate(rho, P)
    nu, shape = len(g), rho.shape
    n = rho.size
    x = np.concatenate([a.ravel() for a in g])

    def F(xv):
        gg = [xv[i * n:(i + 1) * n].reshape(shape) for i in range(nu)]
        return np.concatenate([r.ravel() for r in residual(gg, f, P)])

    nr = math.inf
    for _ in range(max_iter):
        r = F(x)
        nr = max(math.sqrt(float(np.sum(np.abs(r[i * n:(i + 1) * n]) ** 2)) * P.h ** rho.ndim)
                 for i in range(nu))
        if nr <= tol:
            break
        Jm = np.empty((nu * n, nu * n))  # d(residual)/dx by the complex step
        eps = 1e-30
        for j in range(nu * n):
            xc = x.astype(complex)
            xc[j] += 1j * eps
            Jm[:, j] = np.imag(F(xc)) / eps
        x = x - np.linalg.solve(Jm, r)
    g = [x[i * n:(i + 1) * n].reshape(shape) for i in range(nu)]
    return closure(g, rho, P, Emu), g, nr
