"""Plain FP64 CPU oracle of the hydrodynamic PFC scheme in a channel.

TEST INFRASTRUCTURE ONLY, under the same rule as ``oracle.scheme``: only
``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU legs import it;
the product path never does.

The scheme is the one of ``oracle.scheme`` (Sec. 5, Eqs. discrete_a-d, App.
G.2 with the same readings R1-R11), on a 2-D domain periodic in x with walls
at y = 0 and y = L_y (Sec. 6.3: "periodic in the horizontal direction and no
slip moving wall boundary in the vertical direction").  Arrays are [y][x];
the n_y rows are cells j = 0 .. n_y - 1 with centres at (j + 1/2) h, so the
walls lie half a cell outside the first and last rows, and one ghost row on
each side carries the boundary conditions of App. E.2:

  scalars (rho, rho^k, mu, kappa, |u|^2):  phi_{-1} = phi_0            (no flux)
  normal velocity v:                       v_{-1} = -v_0               (no slip)
  tangential velocity u:                   u_{-1} = 2 U_wall - u_0     (no slip,
                                           the wall moving at U_wall, Sec. 6.3)

and the same at the top wall (U_top).  Readings:

W1 The ghost rules are App. E.2's (cell-centred, the wall half a cell out),
   with the tangential rule extended to a moving wall so that the mean of
   the two cells beside the wall is the wall speed.  Sec. 6.3 prints the
   same conditions on boundary nodes; App. E.2's form is the one under which
   the summation-by-parts identities, hence mass conservation and energy
   stability for walls at rest (Thm 5.1), carry over, and it is what the
   pins below check.
W2 Multigrid: x stays nodal (full weighting, injection, linear
   interpolation as in ``oracle.scheme``); y is cell-centred: a coarse cell
   is the union of two fine cells, restriction and injection average the
   two, prolongation interpolates linearly between cell centres (weights
   3/4, 1/4) with the homogeneous ghost rules of a correction.
W3 Products inherit the ghosts of their factors: rho^k v is odd at a wall,
   |u|^2 takes its ghost from the velocity ghosts, (2U - u_0)^2 + v_0^2
   (a Neumann copy only at walls at rest), so plane Couette flow between
   the moving walls is an exact fixed point of the scheme.
W4 The viscous dissipation of App. F counts the wall edges with weight 1/2
   (the summation by parts of sum u Lap_h u with the no-slip ghosts).
Only the local (PFC) functional is supported: the convolution of CDFT has no
wall form in the paper.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

from . import scheme as S

SCAL, UT, VN = 0, 1, 2   # field types: scalar, tangential (x) and normal (y) velocity


@dataclasses.dataclass
class Walls:
    u_bot: float = 0.0   # tangential speed of the wall at y = 0
    u_top: float = 0.0   # tangential speed of the wall at y = L_y

    @staticmethod
    def rest():
        return Walls(0.0, 0.0)


REST = Walls()


def ghost(row, typ, U):
    """Ghost row outside a wall from the adjacent cell row (App. E.2)."""
    if typ == SCAL:
        return row
    if typ == VN:
        return -row
    return 2.0 * U - row


def shx(a, k):
    """Periodic shift along x: result[j, i] = a[j, i + k]."""
    return np.roll(a, -k, axis=1)


def shy(a, k, typ, W=REST):
    """Shift along y with the wall ghosts: result[j, i] = a[j + k, i]."""
    out = np.empty_like(a)
    if k == 1:
        out[:-1] = a[1:]
        out[-1] = ghost(a[-1], typ, W.u_top)
    else:
        out[1:] = a[:-1]
        out[0] = ghost(a[0], typ, W.u_bot)
    return out


def sh(a, d, k, typ, W=REST):
    return shx(a, k) if d == 0 else shy(a, k, typ, W)


def D0(a, d, h, typ, W=REST):
    return (sh(a, d, 1, typ, W) - sh(a, d, -1, typ, W)) / (2.0 * h)


def nb_sum(a, typ, W=REST):
    return shx(a, 1) + shx(a, -1) + shy(a, 1, typ, W) + shy(a, -1, typ, W)


def lap(a, h, typ, W=REST):
    return (nb_sum(a, typ, W) - 4.0 * a) / (h * h)


VEL_T = (UT, VN)


def flux_y(rk, v):
    """y-shifts of the flux rho^k v (reading W3: odd at the walls)."""
    return shy(rk * v, 1, VN), shy(rk * v, -1, VN)


def div_rk(rk, vel, h, W=REST):
    """div_h(rho^k u): the x part periodic, the y part with rho^k Neumann and
    v odd, so the product is odd."""
    u, v = vel
    dx = (shx(rk * u, 1) - shx(rk * u, -1)) / (2.0 * h)
    pv, mv = flux_y(rk, v)
    return dx + (pv - mv) / (2.0 * h)


def D0q(vel, d, h, W=REST):
    """D0 of |u|^2 along d, the wall ghosts of |u|^2 from those of u and v
    (reading W3)."""
    if d == 0:
        q = vel[0] * vel[0] + vel[1] * vel[1]
        return (shx(q, 1) - shx(q, -1)) / (2.0 * h)
    qp = shy(vel[0], 1, UT, W) ** 2 + shy(vel[1], 1, VN, W) ** 2
    qm = shy(vel[0], -1, UT, W) ** 2 + shy(vel[1], -1, VN, W) ** 2
    return (qp - qm) / (2.0 * h)


def vorticity(vel, h, W=REST):
    """omega = D0x v - D0y u with the wall ghosts of u (moving) and v."""
    u, v = vel
    return [D0(v, 0, h, VN, W) - D0(u, 1, h, UT, W)]


def edge_dissipation(vel, h, W=REST):
    """h^2 sum over edges of (D u_c)^2 for both components, the wall edges
    with weight 1/2 (reading W4)."""
    acc = 0.0
    for c, typ in zip(vel, VEL_T):
        Dx = (shx(c, 1) - c) / h
        acc += float(np.sum(Dx * Dx))
        Dy = np.diff(c, axis=0) / h
        acc += float(np.sum(Dy * Dy))
        bot = (c[0] - ghost(c[0], typ, W.u_bot)) / h
        top = (ghost(c[-1], typ, W.u_top) - c[-1]) / h
        acc += 0.5 * float(np.sum(bot * bot) + np.sum(top * top))
    return acc * h * h


# ---------------------------------------------------------------- the scheme
class Coeffs:
    def __init__(self, rk, om):
        self.rk = rk
        self.om = om

    def inject(self):
        return Coeffs(inject(self.rk), [inject(w) for w in self.om])


def apply_N(g, c, P, W):
    """N(g) of ``scheme.apply_N`` (PFC, 2-D) with the wall ghosts."""
    h, s = P.h, P.s
    rho, u, v, mu, kap = g
    vel = [u, v]
    rk = c.rk
    out = [rho + 0.5 * s * div_rk(rk, vel, h, W)]
    wx = S.omega_cross(c.om, vel)
    for a in range(2):
        br = (-0.5 * P.sigma * rk * wx[a] - 0.5 * rk * D0q(vel, a, h, W)
              - rk * D0(mu, a, h, SCAL, W) + 0.5 * P.gamma * lap(vel[a], h, VEL_T[a], W))
        out.append(rk * vel[a] - s * br)
    psi = rho - 1.5
    out.append(mu - psi ** 3 / 3.0 - P.alpha * psi - lap(kap, h, SCAL, W))
    out.append(kap - lap(rho, h, SCAL, W))
    return out


def source(rk, uk, om, P, W):
    h, s = P.h, P.s
    Sx = [rk - 0.5 * s * div_rk(rk, uk, h, W)]
    wx = S.omega_cross(om, uk)
    for a in range(2):
        br = -0.5 * P.sigma * rk * wx[a] + 0.5 * P.gamma * lap(uk[a], h, VEL_T[a], W)
        Sx.append(rk * uk[a] + s * br)
    Sx.append(2.0 * lap(rk, h, SCAL, W))
    Sx.append(np.zeros_like(rk))
    return Sx


def residual(g, f, c, P, W):
    N = apply_N(g, c, P, W)
    return [f[i] - N[i] for i in range(len(f))]


def point_update(g, f, c, P, W, mask):
    """The point block of ``scheme.point_update`` (PFC) with the wall
    ghosts: rho from continuity, kappa, mu with the linearised cubic, the
    2x2 velocity block; projection and damping."""
    h, s = P.h, P.s
    rk = c.rk
    old = [x.copy() for x in g]
    w = P.w_damp
    rho_gs = f[0] - 0.5 * s * div_rk(rk, [g[1], g[2]], h, W)
    rho_gs = np.sqrt(rho_gs * rho_gs + P.delta * P.delta)
    g[0] = np.where(mask, rho_gs, g[0])
    kap_gs = f[4] + lap(g[0], h, SCAL, W)
    g[4] = np.where(mask, kap_gs, g[4])
    phi_old = old[0] - 1.5
    phi_new = g[0] - 1.5
    cubic = phi_old ** 2 * phi_new - (2.0 / 3.0) * phi_old ** 3
    mu_gs = f[3] + cubic + P.alpha * phi_new + lap(g[4], h, SCAL, W)
    g[3] = np.where(mask, mu_gs, g[3])
    vel = [g[1], g[2]]
    # the centre coefficient of Lap_h u at a wall row picks up the odd ghost:
    # u_{-1} = 2U - u_0 puts -u_0 (and 2U) into the neighbour sum
    rhs, diag = [], []
    for a in range(2):
        typ = VEL_T[a]
        nb = nb_sum(vel[a], typ, W)
        # split the neighbour sum into its dependence on the point itself (the
        # ghost mirrors the wall row) and the rest
        self_part = np.zeros_like(rk)
        if typ != SCAL:
            self_part[0] -= vel[a][0]
            self_part[-1] -= vel[a][-1]
        rhs.append(f[1 + a] + s * (-0.5 * rk * D0q(vel, a, h, W) - rk * D0(g[3], a, h, SCAL, W)
                                   + 0.5 * P.gamma * (nb - self_part) / (h * h)))
        d_extra = np.zeros_like(rk)
        d_extra[0] = d_extra[-1] = 1.0  # the mirrored -u_0 moves to the left side
        diag.append(rk + s * P.gamma * 2.0 / (h * h) + 0.5 * s * P.gamma * d_extra / (h * h))
    b = 0.5 * P.sigma * s * rk * c.om[0]
    ax, ay = diag
    det = ax * ay + b * b
    u_gs = (ay * rhs[0] + b * rhs[1]) / det
    v_gs = (ax * rhs[1] - b * rhs[0]) / det
    g[1] = np.where(mask, u_gs, g[1])
    g[2] = np.where(mask, v_gs, g[2])
    comps = range(len(g)) if P.damp_all else [0]
    for i in comps:
        g[i] = np.where(mask, (1.0 - w) * g[i] + w * old[i], g[i])


def smooth(g, f, c, P, W):
    for m in S.color_masks(g[0].shape):
        point_update(g, f, c, P, W, m)


# ------------------------------------------------------- transfers (reading W2)
def inject(a):
    """x: the even nodes; y: the mean of the two fine cells of a coarse cell."""
    return 0.5 * (a[0::2, 0::2] + a[1::2, 0::2])


def restrict(r):
    """x: nodal full weighting; y: the mean of the two fine cells."""
    t = 0.25 * shx(r, -1) + 0.5 * r + 0.25 * shx(r, 1)
    return 0.5 * (t[0::2, 0::2] + t[1::2, 0::2])


def prolong(E, typ):
    """Correction from the coarse to the fine grid: x linear between nodes,
    y linear between cell centres (3/4, 1/4), homogeneous ghosts (a
    correction carries no wall speed)."""
    nyc, nxc = E.shape
    up = np.vstack([ghost(E[:1], typ, 0.0), E[:-1]])       # E_{J-1}
    dn = np.vstack([E[1:], ghost(E[-1:], typ, 0.0)])       # E_{J+1}
    Y = np.empty((2 * nyc, nxc))
    Y[0::2] = 0.75 * E + 0.25 * up
    Y[1::2] = 0.75 * E + 0.25 * dn
    fine = np.zeros((2 * nyc, 2 * nxc))
    fine[:, 0::2] = Y
    fine[:, 1::2] = 0.5 * (Y + np.roll(Y, -1, axis=1))
    return fine


TYPES = (SCAL, UT, VN, SCAL, SCAL)   # rho, u, v, mu, kappa


def can_coarsen(shape, opts):
    ny, nx = shape
    return (nx % 2 == 0 and nx // 2 >= opts.coarsest and (nx // 2) % 2 == 0 and
            ny % 2 == 0 and ny // 2 >= opts.coarsest and (ny // 2) % 2 == 0)


def vcycle(g, f, c, P, W, opts):
    if not can_coarsen(g[0].shape, opts):
        for _ in range(opts.ncoarse):
            smooth(g, f, c, P, W)
        return
    for _ in range(opts.nu1):
        smooth(g, f, c, P, W)
    r = residual(g, f, c, P, W)
    cH = c.inject()
    PH = P.coarse()
    gH = [inject(x) for x in g]
    NH = apply_N(gH, cH, PH, W)
    fH = [NH[i] + restrict(r[i]) for i in range(len(r))]
    gH0 = [x.copy() for x in gH]
    vcycle(gH, fH, cH, PH, W, opts)
    for i in range(len(g)):
        g[i] = g[i] + prolong(gH[i] - gH0[i], TYPES[i])
    for _ in range(opts.nu2):
        smooth(g, f, c, P, W)


def initial_iterate(rk, uk, P, W):
    kap0 = lap(rk, P.h, SCAL, W)
    psi = rk - 1.5
    mu0 = psi ** 3 / 3.0 + P.alpha * psi + lap(kap0, P.h, SCAL, W) + 2.0 * lap(rk, P.h, SCAL, W)
    return [rk.copy(), uk[0].copy(), uk[1].copy(), mu0, kap0]


def closure(g, rk, uk, P, W):
    """Reading R10 with the walls: rho^{k+1} = rho^k - (s/2) div_h(rho^k
    (u^{k+1} + u^k)), projected (the half-sum has the wall speed U)."""
    uh = [0.5 * (g[1] + uk[0]), 0.5 * (g[2] + uk[1])]
    rho = rk - P.s * div_rk(rk, uh, P.h, W)
    return np.sqrt(rho * rho + P.delta * P.delta)


def step(rho, vel, P, W=REST, opts=None):
    """One step with walls.  Returns (rho^{k+1}, [u, v], info)."""
    opts = opts or S.SolverOpts()
    om = vorticity(vel, P.h, W)
    Sx = source(rho, vel, om, P, W)
    c = Coeffs(rho, om)
    g = initial_iterate(rho, vel, P, W)
    hist, cycles = [], 0
    while True:
        nr = S.res_norm(residual(g, Sx, c, P, W), P.h)
        hist.append(nr)
        if not math.isfinite(nr):
            raise S.NoConvergence("non-finite residual")
        if nr <= opts.tol:
            break
        if cycles >= opts.max_cycles:
            raise S.NoConvergence(f"no convergence after {cycles} cycles: {hist}")
        vcycle(g, Sx, c, P, W, opts)
        cycles += 1
    return closure(g, rho, vel, P, W), [g[1].copy(), g[2].copy()], dict(cycles=cycles, hist=hist, g=g, S=Sx, omega=om)


def free_energy(rho, P, W=REST):
    psi = rho - 1.5
    L = lap(rho, P.h, SCAL, W)
    w = P.h * P.h
    return w * float(np.sum(psi ** 4 / 12.0 + 0.5 * P.alpha * psi ** 2 + 0.5 * L * L + rho * L))


def energy(rho, vel, P, W=REST):
    F = free_energy(rho, P, W)
    KE = 0.5 * P.h * P.h * float(np.sum(rho * (vel[0] ** 2 + vel[1] ** 2)))
    return F + KE, F, KE


def solve_dense(rho, vel, P, W=REST, tol=1e-13, max_iter=60):
    """N(g) = S by dense Newton (complex-step Jacobian), no multigrid."""
    om = vorticity(vel, P.h, W)
    Sx = source(rho, vel, om, P, W)
    c = Coeffs(rho, om)
    g = initial_iterate(rho, vel, P, W)
    shape, n = rho.shape, rho.size
    x = np.concatenate([a.ravel() for a in g])

    def F(xv):
        gg = [xv[i * n:(i + 1) * n].reshape(shape) for i in range(5)]
        return np.concatenate([r.ravel() for r in residual(gg, Sx, c, P, W)])

    nr = math.inf
    for _ in range(max_iter):
        r = F(x)
        nr = max(math.sqrt(float(np.sum(np.abs(r[i * n:(i + 1) * n]) ** 2)) * P.h * P.h) for i in range(5))
        if nr <= tol:
            break
        Jm = np.empty((5 * n, 5 * n))
        eps = 1e-30
        for j in range(5 * n):
            xc = x.astype(complex)
            xc[j] += 1j * eps
            Jm[:, j] = np.imag(F(xc)) / eps
        x = x - np.linalg.solve(Jm, r)
    g = [x[i * n:(i + 1) * n].reshape(shape) for i in range(5)]
    return closure(g, rho, vel, P, W), [g[1], g[2]], g, nr
