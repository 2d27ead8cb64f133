"""Plain FP64 CPU oracle of the energy-stable hydrodynamic freezing scheme.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this module.  The
product path (the CUDA library and its Python binding) never imports, calls or
links anything here, and nothing here imports the product path.

What is computed (Baskaran, Guan, Lowengrub, "Energy Stable Multigrid Method
for Local and Non-local Hydrodynamic Models for Freezing"):

* the fully discrete scheme of Sec. 5, Eqs. (discrete_a)-(discrete_d): one
  implicit convex-splitting time step of the compressible Navier-Stokes system
  whose pressure gradient is rho * grad(dF/drho);
* the discrete operators of App. E (centred gradient and divergence, 5-point
  Laplacian, h^d-weighted inner products), periodic boundaries (App. E.2);
* the discrete functionals and their convex splittings: CDFT, Sec. 5.2
  (Eq. CS_DFT_discrete and Lemma 5.2), PFC, Sec. 5.3 (Eq. CS_PFC_discrete and
  Lemma 5.4);
* the non-linear operator N and source S of App. G.1 (CDFT, 3 unknowns per
  point) and App. G.2 (PFC, 5 unknowns per point), derived from the vector
  form of the scheme (readings listed below);
* the solver of Sec. 6 and App. G: FAS multigrid with a point-block damped
  Gauss-Seidel smoother (App. G.1, G.2, G.3) and the positive projection of
  Sec. 6 item 1;
* the convolution kernel of Sec. 6 and the periodic discrete convolution of
  Eq. (discrete_convolution), evaluated by a DFT (numpy.fft as the library
  step) or by the direct O(N^2) sum.

Readings where the paper is silent, garbled or self-contradictory (each one is
also stated where it is used):

R1  vorticity term: the vector form -rho^k omega^k x u^{k+1/2} (Eq. discrete_b)
    is followed; its x-component is +rho omega v.  App. G prints the opposite
    sign.  ``sigma=-1`` reproduces App. G.
R2  the viscous diagonal of the point block carries the factor s
    (a = rho^k + s*gamma*d/h^2); App. G omits it.
R3  the continuity and pressure-term signs are taken from N (Eqs. MGN_*),
    not from the printed smoother formulas.
R4  operator typos of App. E are read as the standard centred operators.
R5  kernel sampling J_{ij} uses the minimum-image distance on the periodic box.
R6  restriction = nodal full weighting, injection of the iterate, bilinear
    prolongation, V-cycle, a fixed number of smoothing sweeps on the coarsest
    grid (the paper defers these to another reference).
R7  damping applies to every unknown of the point block.
R8  projection rho <- sqrt(rho^2 + delta^2) after each point update of rho and
    after the step closure; for delta > 0 (CDFT) also after the coarse-grid
    correction, the other update of rho inside a cycle (Sec. 6 item 1 gives
    the purpose: ln rho must never see a non-positive argument).
R9  residual norm = max over components of sqrt(h^d * sum r^2).
R10 step closure: after the solve, rho^{k+1} is re-evaluated from the
    continuity equation with the final velocity, so mass is exact to round-off.
R11 PFC initial iterate: kappa^0 = Lap_h rho^k, mu^0 = value of the mu
    equation at rho^k.
R12 3-D: 7-point Laplacian, omega = curl_h u (3 components), the 3x3 point block
    a*I + [b]_x.

Arrays are indexed [z][y][x] (3-D) or [y][x] (2-D); direction d = 0 is x
(the last array axis).  All arithmetic is float64.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

PFC = 1
CDFT = 2


# --------------------------------------------------------------------------
# Parameters
# --------------------------------------------------------------------------
@dataclasses.dataclass
class Params:
    """Physical and solver parameters of one level of one problem."""

    kind: int            # PFC or CDFT
    dim: int             # 2 or 3
    h: float             # grid spacing
    s: float             # time step
    gamma: float = 2.0   # viscosity, Sec. 6 ("gamma = 2 in all simulations")
    alpha: float = 0.0   # PFC: alpha = 1 - eps (App. B)
    ce: float = 0.0      # CDFT: (J_e * 1) = h^d sum J_e (Lemma 5.2)
    sigma: float = 1.0   # reading R1
    w_damp: float = 0.5  # App. G.3
    damp_all: bool = True  # reading R7
    delta: float = 0.0   # Sec. 6 item 1 (1e-10 for CDFT, 0 for PFC)

    def coarse(self) -> "Params":
        return dataclasses.replace(self, h=2.0 * self.h)

    @property
    def nvel(self) -> int:
        return self.dim

    @property
    def nunk(self) -> int:
        return 1 + self.dim + (2 if self.kind == PFC else 0)


# --------------------------------------------------------------------------
# Discrete operators, App. E
# --------------------------------------------------------------------------
def sh(a, d, k):
    """Periodic shift: result[p] = a[p + k*e_d] (App. E.2 periodic ghosts)."""
    return np.roll(a, -k, axis=a.ndim - 1 - d)


def D0(a, d, h):
    """Centred difference (phi_{i+1} - phi_{i-1}) / 2h, the component d of
    grad_h (App. E, item 2)."""
    return (sh(a, d, 1) - sh(a, d, -1)) / (2.0 * h)


def lap(a, h):
    """(2d+1)-point Laplacian Delta_h = sum_d d_d(D_d phi) (App. E, item 4)."""
    acc = -2.0 * a.ndim * a
    for d in range(a.ndim):
        acc = acc + sh(a, d, 1) + sh(a, d, -1)
    return acc / (h * h)


def nb_sum(a):
    """Sum of the 2d nearest neighbours (the off-diagonal part of Delta_h)."""
    acc = 0.0
    for d in range(a.ndim):
        acc = acc + sh(a, d, 1) + sh(a, d, -1)
    return acc


def div0(F, h):
    """Centred divergence grad_h . F (App. E, item 3)."""
    return sum(D0(F[d], d, h) for d in range(len(F)))


def vorticity(vel, h):
    """omega^k = grad_h x u^k, Eq. (discrete_d); App. G Eq. (MG_DFT_d) writes
    the 2-D component out.  Returns a list: [omega_z] in 2-D, three
    components in 3-D (reading R12)."""
    if len(vel) == 2:
        u, v = vel
        return [D0(v, 0, h) - D0(u, 1, h)]
    u, v, w = vel
    return [D0(w, 1, h) - D0(v, 2, h),
            D0(u, 2, h) - D0(w, 0, h),
            D0(v, 0, h) - D0(u, 1, h)]


def omega_cross(om, U):
    """omega x U with omega along z in 2-D."""
    if len(U) == 2:
        (w,) = om
        return [-w * U[1], w * U[0]]
    return [om[1] * U[2] - om[2] * U[1],
            om[2] * U[0] - om[0] * U[2],
            om[0] * U[1] - om[1] * U[0]]


def inner(a, b, h):
    """(phi || psi) = h^d sum phi psi (App. E.3)."""
    return float(np.sum(a * b)) * h ** a.ndim


def edge_dissipation(vel, h):
    """sum over velocity components and directions of the edge norms
    [D_d u_c, D_d u_c] = h^d sum (D_d u_c)^2, the viscous dissipation of
    App. F (all four differences in 2-D)."""
    acc = 0.0
    for c in vel:
        for d in range(c.ndim):
            Dd = (sh(c, d, 1) - c) / h
            acc += float(np.sum(Dd * Dd)) * h ** c.ndim
    return acc


# --------------------------------------------------------------------------
# Convolution kernel and discrete convolution, Sec. 6 and Eq.
# (discrete_convolution)
# --------------------------------------------------------------------------
def sample_kernel(shape, h, nu):
    """J, J_e, J_c sampled on the periodic grid (reading R5: minimum image).

    J(x) = sqrt(2) exp(-pi^2 |x|^2 / (2 nu^2)) - exp(-pi^2 |x|^2 / (4 nu^2)),
    J_e = -J where J <= 0 and 0 elsewhere, J_c = J + J_e (Sec. 6)."""
    r2 = np.zeros(shape)
    nd = len(shape)
    for ax in range(nd):
        n = shape[ax]
        k = np.arange(n)
        dist = h * np.minimum(k, n - k)
        bshape = [1] * nd
        bshape[ax] = n
        r2 = r2 + (dist ** 2).reshape(bshape)
    J = math.sqrt(2.0) * np.exp(-math.pi ** 2 * r2 / (2.0 * nu * nu)) \
        - np.exp(-math.pi ** 2 * r2 / (4.0 * nu * nu))
    Je = np.where(J <= 0.0, -J, 0.0)
    Jc = J + Je
    return J, Je, Jc


def conv_fft(J, rho, h):
    """(J * rho)_p = h^d sum_q J_q rho_{p-q}, evaluated by the DFT
    (library step: numpy.fft)."""
    return (h ** rho.ndim) * np.real(np.fft.ifftn(np.fft.fftn(J) * np.fft.fftn(rho)))


def conv_direct(J, rho, h):
    """Direct O(N^2) periodic sum of Eq. (discrete_convolution)."""
    acc = np.zeros_like(rho)
    for q in np.ndindex(*J.shape):
        acc += J[q] * np.roll(rho, q, axis=tuple(range(rho.ndim)))
    return (h ** rho.ndim) * acc


# --------------------------------------------------------------------------
# Discrete functionals and their variational derivatives
# --------------------------------------------------------------------------
def pfc_energy_terms(rho, h, alpha):
    """Discrete PFC free energy, Eq. (CS_PFC_discrete) with reading R4:
    h^d sum [ psi^4/12 + alpha psi^2/2 + (Lap_h rho)^2/2 + rho Lap_h rho ],
    psi = rho - 3/2.  Returns the four terms."""
    psi = rho - 1.5
    L = lap(rho, h)
    w = h ** rho.ndim
    return (w * float(np.sum(psi ** 4)) / 12.0,
            w * alpha * float(np.sum(psi ** 2)) / 2.0,
            w * float(np.sum(L * L)) / 2.0,
            w * float(np.sum(rho * L)))


def pfc_Fc(rho, h, alpha):
    """Convex part, Eq. (CS_PFC_discrete1)."""
    t = pfc_energy_terms(rho, h, alpha)
    return t[0] + t[1] + t[2]


def pfc_Fe(rho, h, alpha):
    """Concave part, Eq. (CS_PFC_discrete2): -(rho || Lap_h rho)."""
    return -pfc_energy_terms(rho, h, alpha)[3]


def pfc_mu_c(rho, h, alpha):
    """delta F_c = psi^3/3 + alpha psi + Lap_h^2 rho (Lemma 5.4)."""
    psi = rho - 1.5
    return psi ** 3 / 3.0 + alpha * psi + lap(lap(rho, h), h)


def pfc_mu_e(rho, h):
    """delta F_e = -2 Lap_h rho (Lemma 5.4)."""
    return -2.0 * lap(rho, h)


def cdft_energy_terms(rho, h, J):
    """Discrete CDFT free energy, Eq. (CS_DFT_discrete):
    F_id = (rho || ln rho - 1), F_ex = -1/2 (rho || J * rho)."""
    w = h ** rho.ndim
    Fid = w * float(np.sum(rho * (np.log(rho) - 1.0)))
    Fex = -0.5 * w * float(np.sum(rho * conv_fft(J, rho, h)))
    return Fid, Fex


def cdft_Fc(rho, h, ce):
    """Eq. (CS_DFT_discrete1)."""
    w = h ** rho.ndim
    return w * float(np.sum(rho * (np.log(rho) - 1.0))) + ce * w * float(np.sum(rho * rho))


def cdft_Fe(rho, h, ce, J):
    """Eq. (CS_DFT_discrete2)."""
    w = h ** rho.ndim
    return ce * w * float(np.sum(rho * rho)) + 0.5 * w * float(np.sum(rho * conv_fft(J, rho, h)))


def cdft_mu_c(rho, ce):
    """delta F_c = ln rho + 2 (J_e*1) rho (Lemma 5.2)."""
    return np.log(rho) + 2.0 * ce * rho


def cdft_mu_e(rho, h, ce, J):
    """delta F_e = 2 (J_e*1) rho + J * rho (Lemma 5.2)."""
    return 2.0 * ce * rho + conv_fft(J, rho, h)


# --------------------------------------------------------------------------
# Non-linear operator N and source S (App. G), from the vector scheme
# --------------------------------------------------------------------------
class Coeffs:
    """Per-level coefficients of N: rho^k and omega^k (and, on the finest
    level only, what enters S)."""

    def __init__(self, rk, om):
        self.rk = rk
        self.om = om

    def inject(self):
        return Coeffs(inject(self.rk), [inject(w) for w in self.om])


def apply_N(g, c: Coeffs, P: Params):
    """N(g) for g = (rho, u_1..u_d[, mu, kappa]).

    Continuity (Eq. MGN_*_a): rho + (s/2) div_h(rho^k u).
    Momentum (Eq. MGN_*_b,c, with readings R1, R3):
        rho^k u - s[ -(sigma/2) rho^k (omega^k x u) - (rho^k/2) grad_h |u|^2
                     - rho^k grad_h mu_impl + (gamma/2) Lap_h u ],
    where mu_impl = mu (PFC unknown) or ln rho + 2 c_e rho (CDFT).
    PFC (Eqs. MGN_PFC_d,e): mu - psi^3/3 - alpha psi - Lap_h kappa and
    kappa - Lap_h rho.
    Written with plain products so that a complex step can differentiate it.
    """
    d, h, s = P.dim, P.h, P.s
    rho = g[0]
    vel = g[1:1 + d]
    rk = c.rk
    out = [rho + 0.5 * s * div0([rk * vel[a] for a in range(d)], h)]
    q = sum(vel[a] * vel[a] for a in range(d))
    if P.kind == PFC:
        m = g[1 + d]
    else:
        m = np.log(rho) + 2.0 * P.ce * rho
    wx = omega_cross(c.om, vel)
    for a in range(d):
        br = (-0.5 * P.sigma * rk * wx[a] - 0.5 * rk * D0(q, a, h)
              - rk * D0(m, a, h) + 0.5 * P.gamma * lap(vel[a], h))
        out.append(rk * vel[a] - s * br)
    if P.kind == PFC:
        mu, kap = g[1 + d], g[2 + d]
        psi = rho - 1.5
        out.append(mu - psi ** 3 / 3.0 - P.alpha * psi - lap(kap, h))
        out.append(kap - lap(rho, h))
    return out


def source(rk, uk, om, P: Params, C=None):
    """S of App. G (Eqs. MGS_DFT_a-c, MGS_PFC_a-e): the explicit halves of
    u^{k+1/2}, the explicit part of mu (2 Lap_h rho^k for PFC;
    2 c_e rho^k + J*rho^k for CDFT, entering through -rho^k grad_h mu)."""
    d, h, s = P.dim, P.h, P.s
    S = [rk - 0.5 * s * div0([rk * uk[a] for a in range(d)], h)]
    wx = omega_cross(om, uk)
    for a in range(d):
        br = -0.5 * P.sigma * rk * wx[a] + 0.5 * P.gamma * lap(uk[a], h)
        if P.kind == CDFT:
            br = br + rk * D0(2.0 * P.ce * rk + C, a, h)
        S.append(rk * uk[a] + s * br)
    if P.kind == PFC:
        S.append(2.0 * lap(rk, h))
        S.append(np.zeros_like(rk))
    return S


def residual(g, S, c, P):
    N = apply_N(g, c, P)
    return [S[i] - N[i] for i in range(len(S))]


def res_norm(r, h):
    """Reading R9: max over components of sqrt(h^d sum r^2)."""
    return max(math.sqrt(float(np.sum(x * x)) * h ** x.ndim) for x in r)


# --------------------------------------------------------------------------
# Point-block damped Gauss-Seidel smoother (App. G.1, G.2, G.3)
# --------------------------------------------------------------------------
def color_masks(shape):
    idx = np.indices(shape).sum(axis=0)
    return [(idx % 2) == 0, (idx % 2) == 1]


def point_update(g, S, c: Coeffs, P: Params, mask):
    """Solve the point block of N(g) = S at the points of ``mask`` with all
    other points held fixed, then project rho and damp.

    No two points of ``mask`` may be neighbours (one colour, or one point).
    In the point block the unknowns decouple into a triangular chain
    (App. G: the continuity row has no u_ij, the momentum rows no mu_ij):
      rho   from continuity (neighbour velocities), then projection (Sec. 6);
      kappa from N5 with the new rho_ij            (PFC);
      mu    from N4 with the cubic linearised about the previous rho_ij,
            (phi^{l+1})^3 ~ 3 (phi^l)^2 phi^{l+1} - 2 (phi^l)^3 (App. G.2);
      (u_1..u_d) from the d x d block a I + [b]_x, a = rho^k + s gamma d/h^2
            (reading R2), b = (sigma s/2) rho^k omega^k.
    """
    d, h, s = P.dim, P.h, P.s
    rk = c.rk
    old = [x.copy() for x in g]
    w = P.w_damp

    # rho from the continuity equation
    rho_gs = S[0] - 0.5 * s * div0([rk * g[1 + a] for a in range(d)], h)
    rho_gs = np.sqrt(rho_gs * rho_gs + P.delta * P.delta)
    g[0] = np.where(mask, rho_gs, g[0])

    if P.kind == PFC:
        # kappa = S5 + Lap_h rho (new rho_ij)
        kap_gs = S[2 + d] + lap(g[0], h)
        g[2 + d] = np.where(mask, kap_gs, g[2 + d])
        # mu with the linearised cubic
        phi_old = old[0] - 1.5
        phi_new = g[0] - 1.5
        cubic = phi_old ** 2 * phi_new - (2.0 / 3.0) * phi_old ** 3
        mu_gs = S[1 + d] + cubic + P.alpha * phi_new + lap(g[2 + d], h)
        g[1 + d] = np.where(mask, mu_gs, g[1 + d])
        m = g[1 + d]
    else:
        m = np.log(g[0]) + 2.0 * P.ce * g[0]

    vel = g[1:1 + d]
    q = sum(vel[a] * vel[a] for a in range(d))
    a_diag = rk + s * P.gamma * d / (h * h)
    rhs = []
    for a in range(d):
        rhs.append(S[1 + a] + s * (-0.5 * rk * D0(q, a, h) - rk * D0(m, a, h)
                                   + 0.5 * P.gamma * nb_sum(vel[a]) / (h * h)))
    bco = [0.5 * P.sigma * s * rk * wz for wz in c.om]
    if d == 2:
        (b,) = bco
        det = a_diag * a_diag + b * b
        u_gs = (a_diag * rhs[0] + b * rhs[1]) / det
        v_gs = (a_diag * rhs[1] - b * rhs[0]) / det
        new_vel = [u_gs, v_gs]
    else:
        # (a I + [b]_x)^{-1} y = (a^2 y - a b x y + (b.y) b) / (a (a^2 + |b|^2))
        bx = omega_cross(bco, rhs)
        bdy = sum(bco[i] * rhs[i] for i in range(3))
        den = a_diag * (a_diag * a_diag + sum(bi * bi for bi in bco))
        new_vel = [(a_diag * a_diag * rhs[i] - a_diag * bx[i] + bdy * bco[i]) / den
                   for i in range(3)]
    for a in range(d):
        g[1 + a] = np.where(mask, new_vel[a], g[1 + a])

    # damping (App. G.3, reading R7)
    comps = range(len(g)) if P.damp_all else [0]
    for i in comps:
        g[i] = np.where(mask, (1.0 - w) * g[i] + w * old[i], g[i])


def smooth(g, S, c, P, ordering="redblack"):
    """One smoothing iteration: red then black half sweeps, or a
    lexicographic sweep (x fastest) as printed in App. G."""
    if ordering == "redblack":
        for m in color_masks(g[0].shape):
            point_update(g, S, c, P, m)
    else:
        shape = g[0].shape
        for p in np.ndindex(*shape):
            m = np.zeros(shape, dtype=bool)
            m[p] = True
            point_update(g, S, c, P, m)


# --------------------------------------------------------------------------
# Grid transfers (reading R6) and the FAS V-cycle (Sec. 6)
# --------------------------------------------------------------------------
def inject(a):
    return a[tuple(slice(None, None, 2) for _ in range(a.ndim))].copy()


def restrict_fw(r):
    """Nodal full weighting: [1/4 1/2 1/4] along every axis, then injection."""
    t = r
    for d in range(r.ndim):
        t = 0.25 * sh(t, d, -1) + 0.5 * t + 0.25 * sh(t, d, 1)
    return inject(t)


def prolong(E):
    """Bilinear (trilinear) interpolation from the coarse to the fine grid."""
    fine = np.zeros(tuple(2 * n for n in E.shape))
    fine[tuple(slice(None, None, 2) for _ in range(E.ndim))] = E
    for d in range(E.ndim):
        fine = 0.5 * sh(fine, d, -1) + fine + 0.5 * sh(fine, d, 1)
    return fine


@dataclasses.dataclass
class SolverOpts:
    nu1: int = 2
    nu2: int = 2
    coarsest: int = 4
    ncoarse: int = 20
    tol: float = 1e-10
    max_cycles: int = 60
    ordering: str = "redblack"


def can_coarsen(shape, opts):
    """Coarsen while every size halves to an even size >= ``coarsest``
    (red-black ordering needs even periodic sizes on every level)."""
    return all(n % 2 == 0 and n // 2 >= opts.coarsest and (n // 2) % 2 == 0 for n in shape)


def vcycle(g, f, c, P, opts):
    """FAS V(nu1, nu2) cycle on N(g) = f (standard FAS, Sec. 6)."""
    if not can_coarsen(g[0].shape, opts):
        for _ in range(opts.ncoarse):
            smooth(g, f, c, P, opts.ordering)
        return
    for _ in range(opts.nu1):
        smooth(g, f, c, P, opts.ordering)
    r = residual(g, f, c, P)
    cH = c.inject()
    PH = P.coarse()
    gH = [inject(x) for x in g]
    NH = apply_N(gH, cH, PH)
    fH = [NH[i] + restrict_fw(r[i]) for i in range(len(r))]
    gH0 = [x.copy() for x in gH]
    vcycle(gH, fH, cH, PH, opts)
    for i in range(len(g)):
        g[i] = g[i] + prolong(gH[i] - gH0[i])
    if P.delta > 0.0:
        # reading R8: the corrected density is projected before ln rho is
        # evaluated on it again (Sec. 6 item 1)
        g[0] = np.sqrt(g[0] * g[0] + P.delta * P.delta)
    for _ in range(opts.nu2):
        smooth(g, f, c, P, opts.ordering)


class NoConvergence(RuntimeError):
    pass


def initial_iterate(rk, uk, P):
    """g^0 = (rho^k, u^k[, mu^0, kappa^0]) with reading R11."""
    g = [rk.copy()] + [x.copy() for x in uk]
    if P.kind == PFC:
        kap0 = lap(rk, P.h)
        psi = rk - 1.5
        mu0 = psi ** 3 / 3.0 + P.alpha * psi + lap(kap0, P.h) + 2.0 * lap(rk, P.h)
        g += [mu0, kap0]
    return g


def closure(g, rk, uk, P):
    """Reading R10: rho^{k+1} = rho^k - (s/2) div_h(rho^k u^{k+1/2}) with the
    final velocity, then the projection of Sec. 6."""
    d = P.dim
    uh = [0.5 * (g[1 + a] + uk[a]) for a in range(d)]
    rho = rk - P.s * div0([rk * uh[a] for a in range(d)], P.h)
    return np.sqrt(rho * rho + P.delta * P.delta)


def step(rho, vel, P: Params, opts: SolverOpts = None, J=None, g0=None):
    """Advance (rho^k, u^k) by one time step of size P.s.

    Returns (rho^{k+1}, [u^{k+1}...], info) where info holds the V-cycle
    count, the residual history, the converged iterate g (PFC: with mu and
    kappa) and the explicit inputs (omega^k, S, J*rho^k)."""
    opts = opts or SolverOpts()
    om = vorticity(vel, P.h)
    C = conv_fft(J, rho, P.h) if P.kind == CDFT else None
    S = source(rho, vel, om, P, C)
    c = Coeffs(rho, om)
    g = initial_iterate(rho, vel, P) if g0 is None else [x.copy() for x in g0]
    hist = []
    cycles = 0
    while True:
        r = residual(g, S, c, P)
        nr = res_norm(r, P.h)
        hist.append(nr)
        if not math.isfinite(nr):
            raise NoConvergence("non-finite residual")
        if nr <= opts.tol:
            break
        if cycles >= opts.max_cycles:
            raise NoConvergence(f"no convergence after {cycles} cycles: {hist}")
        vcycle(g, S, c, P, opts)
        cycles += 1
    rho_new = closure(g, rho, vel, P)
    info = dict(cycles=cycles, hist=hist, g=g, omega=om, S=S, C=C)
    return rho_new, [x.copy() for x in g[1:1 + P.dim]], info


# --------------------------------------------------------------------------
# Energy and mass (Thm 5.1)
# --------------------------------------------------------------------------
def kinetic(rho, vel, h):
    """KE = 1/2 (rho u || u)."""
    return 0.5 * sum(inner(rho * u, u, h) for u in vel)


def free_energy(rho, P: Params, J=None):
    if P.kind == PFC:
        return sum(pfc_energy_terms(rho, P.h, P.alpha))
    return sum(cdft_energy_terms(rho, P.h, J))


def energy(rho, vel, P: Params, J=None):
    """(E, F, KE) with E = 1/2 (rho u || u) + F[rho] (Thm 5.1)."""
    F = free_energy(rho, P, J)
    KE = kinetic(rho, vel, P.h)
    return F + KE, F, KE


def mass(rho, h):
    """(rho || 1)."""
    return float(np.sum(rho)) * h ** rho.ndim


def cdft_setup(shape, h, nu):
    """J and c_e = (J_e * 1) = h^d sum J_e for a CDFT problem."""
    J, Je, _ = sample_kernel(shape, h, nu)
    ce = float(np.sum(Je)) * h ** len(shape)
    return J, ce
