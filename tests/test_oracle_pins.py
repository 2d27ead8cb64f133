"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: discrete
symbols of the stencils, closed-form integrals and sums, the invariants of
Thm 5.1 and Lemmas 5.2/5.4, a linearised closed-form step, a dense Newton
solve, and the refinement order of Sec. 6.1.
"""
import math

import numpy as np
import pytest

from oracle import newton
from oracle import scheme as S
from paper_1503_07416_gb300 import inputs

RNG = np.random.default_rng(12345)


def pfc_params(h, s, alpha=0.975, **kw):
    return S.Params(kind=S.PFC, dim=2, h=h, s=s, alpha=alpha, **kw)


def cdft_params(shape, h, s, nu, **kw):
    J, ce = S.cdft_setup(shape, h, nu)
    return S.Params(kind=S.CDFT, dim=2, h=h, s=s, ce=ce, delta=1e-10, **kw), J


def mode(n, h, m, axis=0):
    x = np.arange(n) * h
    X, Y = np.meshgrid(x, x, indexing="xy")
    k = 2 * math.pi * m / (n * h)
    return (X if axis == 0 else Y), k


# ---------------------------------------------------------------- operators
def test_stencil_symbols():
    """App. E: D0 sin(kx) = (sin kh / h) cos(kx); Lap_h cos(kx) =
    -(4/h^2) sin^2(kh/2) cos(kx), along x and along y."""
    n, h = 32, 0.7
    for axis in (0, 1):
        X, k = mode(n, h, 3, axis)
        d0 = S.D0(np.sin(k * X), axis, h)
        assert np.allclose(d0, math.sin(k * h) / h * np.cos(k * X), atol=1e-13)
        lp = S.lap(np.cos(k * X), h)
        lam = -4.0 / h ** 2 * math.sin(k * h / 2) ** 2
        assert np.allclose(lp, lam * np.cos(k * X), atol=1e-12)


def test_vorticity_of_rigid_modes():
    """omega = dv/dx - du/dy: for u = -sin(ky), v = sin(kx) the centred curl is
    (sin kh/h)(cos kx + cos ky)."""
    n, h = 32, 0.5
    X, k = mode(n, h, 2, 0)
    Y, _ = mode(n, h, 2, 1)
    u, v = -np.sin(k * Y), np.sin(k * X)
    (w,) = S.vorticity([u, v], h)
    assert np.allclose(w, math.sin(k * h) / h * (np.cos(k * X) + np.cos(k * Y)), atol=1e-13)


def test_transfers():
    """Nodal full weighting keeps constants, bilinear prolongation keeps
    constants and linear-in-index data, and FW = 2^-d P^T (adjointness)."""
    n = 16
    c = np.full((n, n), 3.25)
    assert np.allclose(S.restrict_fw(c), 3.25)
    assert np.allclose(S.prolong(np.full((8, 8), 3.25)), 3.25)
    E = RNG.standard_normal((8, 8))
    fine = S.prolong(E)
    assert np.array_equal(fine[::2, ::2], E)
    assert np.allclose(fine[::2, 1:-1:2], 0.5 * (E[:, :-1] + E[:, 1:]))
    r = RNG.standard_normal((n, n))
    lhs = np.sum(S.restrict_fw(r) * E) * 4.0
    rhs = np.sum(r * S.prolong(E))
    assert abs(lhs - rhs) < 1e-12


# ---------------------------------------------------------------- convolution
def test_conv_fft_equals_direct_sum():
    """DFT evaluation equals the O(N^2) sum of Eq. (discrete_convolution)."""
    for n in (4, 8, 16):
        h = 34.0 / n
        J, _, _ = S.sample_kernel((n, n), h, 2.362)
        rho = RNG.uniform(0.2, 0.4, (n, n))
        a = S.conv_fft(J, rho, h)
        b = S.conv_direct(J, rho, h)
        assert np.max(np.abs(a - b)) <= 1e-14 * np.max(np.abs(b)) * n


def test_kernel_integral_and_symbol_closed_form():
    """h^2 sum J -> int J = (2 sqrt2 - 4) nu^2 / pi < 0 (Sec. 2.1 requires
    int J < 0), and J * cos(k.x) = Jhat(k) cos(k.x) with the Gaussian Fourier
    transform Jhat(k) = (2 sqrt2 nu^2/pi) e^{-k^2 nu^2/(2 pi^2)}
    - (4 nu^2/pi) e^{-k^2 nu^2/pi^2}."""
    n, h, nu = 256, 17.0 / 128, 2.362
    J, Je, Jc = S.sample_kernel((n, n), h, nu)
    integral = float(np.sum(J)) * h * h
    exact = (2 * math.sqrt(2) - 4) * nu ** 2 / math.pi
    assert exact < 0
    assert abs(integral - exact) < 1e-11 * abs(exact)
    assert np.all(Je >= 0) and np.all(Jc >= 0) and np.allclose(Jc - Je, J)
    for m in (1, 5, 17):
        X, k = mode(n, h, m, 0)
        c = S.conv_fft(J, np.cos(k * X), h)
        jh = (2 * math.sqrt(2) * nu ** 2 / math.pi) * math.exp(-k * k * nu * nu / (2 * math.pi ** 2)) \
            - (4 * nu ** 2 / math.pi) * math.exp(-k * k * nu * nu / math.pi ** 2)
        assert np.allclose(c, jh * np.cos(k * X), atol=1e-11)


def test_ce_closed_form():
    """c_e = (J_e * 1) = h^2 sum J_e tends to int J_e = sqrt(2) nu^2 / pi:
    J < 0 exactly where |x|^2 > 2 nu^2 ln 2 / pi^2, and the two Gaussian tails
    beyond that radius integrate in closed form.  J_e has a kink there, so
    the grid sum converges at O(h^2)."""
    nu = 2.362
    exact = math.sqrt(2.0) * nu * nu / math.pi
    errs = []
    for n in (128, 256):
        h = 34.0 / n
        J, ce = S.cdft_setup((n, n), h, nu)
        errs.append(abs(ce - exact))
    assert errs[1] < 5e-3 * exact
    assert errs[1] < errs[0]


def test_cdft_convexity_bound():
    """Lemma 5.2 needs F_e convex: 2 c_e + Jhat(k) >= 0 for every k, with
    c_e = h^2 sum J_e; the minimum is bounded below by -Jhat(0) > 0."""
    n, h, nu = 128, 17.0 / 128, 2.362
    J, Je, _ = S.sample_kernel((n, n), h, nu)
    ce = float(np.sum(Je)) * h * h
    Jhat = np.real(np.fft.fft2(J)) * h * h
    assert np.min(2 * ce + Jhat) >= -Jhat[0, 0] - 1e-12
    assert -Jhat[0, 0] > 0


# ---------------------------------------------------------------- functionals
def test_pfc_energy_of_a_mode():
    """For rho = 3/2 + A cos(kx) on a grid with 4k below Nyquist, the discrete
    sums of cos^2 and cos^4 are N/2 and 3N/8, and Lap_h acts by its symbol, so
    F = h^2 N [A^4/32 + alpha A^2/4 + lam^2 A^2/4 + lam A^2/2]."""
    n, h, A, alpha = 64, 0.5, 0.3, 0.975
    X, k = mode(n, h, 3, 0)
    rho = 1.5 + A * np.cos(k * X)
    lam = -4.0 / h ** 2 * math.sin(k * h / 2) ** 2
    exact = h * h * n * n * (A ** 4 / 32 + alpha * A * A / 4 + lam * lam * A * A / 4 + lam * A * A / 2)
    got = sum(S.pfc_energy_terms(rho, h, alpha))
    assert abs(got - exact) < 1e-12 * abs(exact) * 100


def test_cdft_energy_uniform():
    """Uniform rho: F_id = |Omega| rho (ln rho - 1), F_ex = -1/2 |Omega| rho^2 Jhat(0)."""
    n, h, nu, rb = 32, 17.0 / 32, 2.362, 0.1 * math.pi
    J, _, _ = S.sample_kernel((n, n), h, nu)
    Fid, Fex = S.cdft_energy_terms(np.full((n, n), rb), h, J)
    area = (n * h) ** 2
    assert abs(Fid - area * rb * (math.log(rb) - 1)) < 1e-12 * abs(Fid)
    assert abs(Fex + 0.5 * area * rb * rb * float(np.sum(J)) * h * h) < 1e-12 * abs(Fex)


@pytest.mark.parametrize("kind", ["pfc", "cdft"])
def test_mu_is_gradient_of_split_energies(kind):
    """delta F_c and delta F_e of Lemmas 5.2/5.4 are the gradients of F_c and
    F_e in the (.||.) inner product: central directional differences."""
    n, h = 16, 0.6
    rho = RNG.uniform(0.3, 0.5, (n, n)) + (1.0 if kind == "pfc" else 0.0)
    eta = RNG.standard_normal((n, n))
    eps = 1e-5
    if kind == "pfc":
        a = 0.7
        fc = lambda r: S.pfc_Fc(r, h, a)
        fe = lambda r: S.pfc_Fe(r, h, a)
        gc, ge = S.pfc_mu_c(rho, h, a), S.pfc_mu_e(rho, h)
    else:
        J, ce = S.cdft_setup((n, n), h, 2.362)
        fc = lambda r: S.cdft_Fc(r, h, ce)
        fe = lambda r: S.cdft_Fe(r, h, ce, J)
        gc, ge = S.cdft_mu_c(rho, ce), S.cdft_mu_e(rho, h, ce, J)
    for f, g in ((fc, gc), (fe, ge)):
        dd = (f(rho + eps * eta) - f(rho - eps * eta)) / (2 * eps)
        assert abs(dd - S.inner(g, eta, h)) < 1e-7 * max(1.0, abs(dd))


@pytest.mark.parametrize("kind", ["pfc", "cdft"])
def test_convex_splitting_inequality(kind):
    """Eq. (ineq2c): F(phi) - F(psi) <= (dF_c(phi) - dF_e(psi) || phi - psi)
    for arbitrary pairs (Lemmas 5.2, 5.4)."""
    n, h = 16, 0.6
    for _ in range(20):
        base = 1.0 if kind == "pfc" else 0.0
        phi = base + RNG.uniform(0.1, 0.8, (n, n))
        psi = base + RNG.uniform(0.1, 0.8, (n, n))
        if kind == "pfc":
            a = 0.6
            F = lambda r: S.pfc_Fc(r, h, a) - S.pfc_Fe(r, h, a)
            rhs = S.inner(S.pfc_mu_c(phi, h, a) - S.pfc_mu_e(psi, h), phi - psi, h)
        else:
            J, ce = S.cdft_setup((n, n), h, 2.362)
            F = lambda r: sum(S.cdft_energy_terms(r, h, J))
            rhs = S.inner(S.cdft_mu_c(phi, ce) - S.cdft_mu_e(psi, h, ce, J), phi - psi, h)
        assert F(phi) - F(psi) <= rhs + 1e-10 * abs(rhs)


# ---------------------------------------------------------------- the scheme
def _linear_mode_prediction(kind, rb, a, b, k, h, s, gamma, alpha=None, ce=None, jhat=None):
    """One step of Eqs. (discrete_a-c) linearised about (rho_bar, 0) for
    rho^k = rho_bar + a cos(kx), u^k = b sin(kx): with the discrete symbols
    s1 = sin(kh)/h of D0 and lam of Lap_h, mu^{k+1} = c1 A + c0 a, and
        (A - a) + s rho_bar s1 (B + b)/2 = 0,
        rho_bar (B - b) = s [rho_bar s1 mu' + gamma lam (B + b)/2]."""
    s1 = math.sin(k * h) / h
    lam = -4.0 / h ** 2 * math.sin(k * h / 2) ** 2
    if kind == "pfc":
        psi = rb - 1.5
        c1 = psi * psi + alpha + lam * lam
        c0 = 2 * lam
    else:
        c1 = 1.0 / rb + 2 * ce
        c0 = -2 * ce - jhat
    M = np.array([[1.0, s * rb * s1 / 2],
                  [-s * rb * s1 * c1, rb - s * gamma * lam / 2]])
    rhs = np.array([a - s * rb * s1 * b / 2,
                    rb * b + s * rb * s1 * c0 * a + s * gamma * lam * b / 2])
    return np.linalg.solve(M, rhs)


@pytest.mark.parametrize("kind", ["pfc", "cdft"])
@pytest.mark.parametrize("axis", [0, 1])
def test_linearised_single_mode_step(kind, axis):
    """A small single Fourier mode evolves by the closed-form 2x2
    amplification of the linearised scheme (to O(delta^2))."""
    n = 32
    if kind == "pfc":
        h, s, rb = 0.5, 0.05, 1.5 - 0.07 * math.sqrt(3)
        P = pfc_params(h, s, alpha=0.975)
        J = None
    else:
        h, s, rb = 17.0 / 64, 0.05, 0.1 * math.pi
        P, J = cdft_params((n, n), h, s, 2.362)
    X, k = mode(n, h, 2, axis)
    delta = 1e-6
    a, b = delta, 0.7 * delta
    rho = rb + a * np.cos(k * X)
    vel = [np.zeros((n, n)), np.zeros((n, n))]
    vel[axis] = b * np.sin(k * X)
    jhat = float(np.sum(J * np.cos(k * mode(n, h, 2, 0)[0]))) * h * h if J is not None else None
    A, B = _linear_mode_prediction(kind, rb, a, b, k, h, s, P.gamma, alpha=P.alpha, ce=P.ce, jhat=jhat)
    r1, v1, info = S.step(rho, vel, P, S.SolverOpts(tol=1e-13, max_cycles=80), J=J)
    got_A = 2 * np.mean((r1 - rb) * np.cos(k * X))
    got_B = 2 * np.mean(v1[axis] * np.sin(k * X))
    assert abs(got_A - A) < 1e-4 * abs(A)
    assert abs(got_B - B) < 1e-4 * abs(B)
    assert np.max(np.abs(v1[1 - axis])) < 1e-3 * abs(B)


def test_shear_flow_generates_no_cross_flow():
    """For the parallel shear u = (0, V cos(kx)), u.grad u = 0 while the scheme
    splits it as omega x u + grad|u|^2/2 (Sec. 4).  With the vector-form sign
    the two discrete terms cancel up to truncation, so the x-velocity after
    one step is far below the s V^2 k scale that a sign error produces."""
    n, h, s, V = 64, 0.5, 0.01, 1e-3
    X, k = mode(n, h, 1, 0)
    rb = 1.5 - 0.07 * math.sqrt(3)
    rho = np.full((n, n), rb)
    vel = [np.zeros((n, n)), V * np.cos(k * X)]
    out = {}
    for sig in (1.0, -1.0):
        P = pfc_params(h, s, sigma=sig)
        _, v1, _ = S.step(rho, vel, P, S.SolverOpts(tol=1e-12))
        out[sig] = np.max(np.abs(v1[0]))
    scale = s * V * V * k
    assert out[-1.0] > 0.5 * scale
    assert out[1.0] < 0.05 * scale


SHEAR_3D = [(0, 1), (1, 0), (0, 2), (2, 0), (1, 2), (2, 1)]


@pytest.mark.parametrize("a,b", SHEAR_3D)
def test_3d_shear_flow_generates_no_cross_flow(a, b):
    """3-D analogue of the shear pin (Sec. 4 identity u.grad u = omega x u +
    grad|u|^2/2, Eq. discrete_b): u_a = V cos(k x_b), the other components
    zero, has u.grad u = 0.  Its centred curl has one component, along the
    third axis, and omega x u points along x_b, where grad|u|^2/2 cancels it
    only with the vector-form sign.  The six (a, b) pairs exercise every
    component of the 3-D curl and every slot of the cross product; a sign
    error in any of them drives a cross flow of the s V^2 k scale."""
    n, h, s, V = 16, 0.5, 0.01, 1e-3
    rb = 1.5 - 0.07 * math.sqrt(3)
    k = 2 * math.pi / (n * h)
    shape = (n, n, n)
    bshape = [1, 1, 1]
    bshape[2 - b] = n
    prof = V * np.cos(k * np.arange(n) * h).reshape(bshape) * np.ones(shape)
    out = {}
    for sig in (1.0, -1.0):
        P = S.Params(kind=S.PFC, dim=3, h=h, s=s, alpha=0.975, sigma=sig)
        vel = [np.zeros(shape) for _ in range(3)]
        vel[a] = prof.copy()
        _, v1, _ = S.step(np.full(shape, rb), vel, P, S.SolverOpts(tol=1e-12, coarsest=2))
        out[sig] = max(float(np.max(np.abs(v1[c]))) for c in range(3) if c != a)
    scale = s * V * V * k
    assert out[-1.0] > 0.5 * scale, out
    assert out[1.0] < 0.1 * scale, out


def test_3d_kinetic_energy_identity():
    """The exact discrete identity of App. F in 3-D:
    KE^{k+1} - KE^k + (rho^{k+1} - rho^k || mu^{k+1}) + s gamma D = 0, with D
    the edge norms of all nine differences D_d u_c of u^{k+1/2}; the energy
    drop is at least s gamma D."""
    n = 8
    rng = np.random.default_rng(19)
    rho = 0.8 + 0.05 * rng.uniform(-1, 1, (n, n, n))
    vel = [0.05 * rng.standard_normal((n, n, n)) for _ in range(3)]
    P = S.Params(kind=S.PFC, dim=3, h=0.9, s=0.02, alpha=0.6)
    for _ in range(2):
        E0, _, K0 = S.energy(rho, vel, P)
        r1, v1, info = S.step(rho, vel, P, S.SolverOpts(tol=1e-13, coarsest=2))
        E1, _, K1 = S.energy(r1, v1, P)
        mu = info["g"][4]
        uh = [0.5 * (x + y) for x, y in zip(v1, vel)]
        D = S.edge_dissipation(uh, P.h)
        ident = K1 - K0 + S.inner(r1 - rho, mu, P.h) + P.s * P.gamma * D
        assert abs(ident) < 1e-10 * max(1.0, abs(E0)), ident
        assert E1 - E0 <= -P.s * P.gamma * D + 1e-10
        rho, vel = r1, v1


@pytest.mark.parametrize("kind", ["pfc", "cdft"])
def test_uniform_state_is_a_fixed_point(kind):
    """rho = rho_bar, u = 0 makes every difference vanish: zero V-cycles and
    the same state back."""
    n = 16
    if kind == "pfc":
        P, J, rb = pfc_params(0.5, 0.01), None, 1.3787
    else:
        (P, J), rb = cdft_params((n, n), 17.0 / 32, 0.02, 2.362), 0.1 * math.pi
    rho = np.full((n, n), rb)
    vel = [np.zeros((n, n)), np.zeros((n, n))]
    r1, v1, info = S.step(rho, vel, P, S.SolverOpts(tol=1e-12), J=J)
    assert info["cycles"] == 0
    assert np.array_equal(r1, rho)
    assert all(np.array_equal(a, b) for a, b in zip(v1, vel))


def _random_state(kind, n, seed):
    rng = np.random.default_rng(seed)
    if kind == "pfc":
        rho = 1.37 + 0.05 * rng.uniform(-1, 1, (n, n))
    else:
        rho = 0.1 * math.pi * (1 + 0.1 * rng.uniform(0, 1, (n, n)))
    vel = [0.05 * rng.standard_normal((n, n)), 0.05 * rng.standard_normal((n, n))]
    return rho, vel


@pytest.mark.parametrize("kind", ["pfc", "cdft"])
def test_mass_energy_and_kinetic_identity(kind):
    """Thm 5.1: (rho^{k+1}||1) = (rho^k||1) to round-off and E^{k+1} <= E^k;
    the proof (App. F) gives the exact identity
    KE^{k+1} - KE^k + (rho^{k+1} - rho^k || mu^{k+1}) + s gamma D = 0,
    D = sum of the edge norms of D_x, D_y of both components of u^{k+1/2}."""
    n = 32
    rho, vel = _random_state(kind, n, 7)
    if kind == "pfc":
        P, J = pfc_params(0.5, 0.01), None
    else:
        P, J = cdft_params((n, n), 17.0 / 32, 0.02, 2.362)
    M0 = S.mass(rho, P.h)
    for _ in range(4):
        E0, F0, K0 = S.energy(rho, vel, P, J)
        r1, v1, info = S.step(rho, vel, P, S.SolverOpts(tol=1e-12), J=J)
        E1, F1, K1 = S.energy(r1, v1, P, J)
        assert abs(S.mass(r1, P.h) - M0) < 1e-13 * n * n * abs(M0) / 100
        assert E1 <= E0 + 1e-11
        if kind == "pfc":
            mu = info["g"][3]
        else:
            mu = S.cdft_mu_c(r1, P.ce) - S.cdft_mu_e(rho, P.h, P.ce, J)
        uh = [0.5 * (a + b) for a, b in zip(v1, vel)]
        ident = K1 - K0 + S.inner(r1 - rho, mu, P.h) + P.s * P.gamma * S.edge_dissipation(uh, P.h)
        assert abs(ident) < 1e-9 * max(1.0, abs(E0))
        # sharper: the energy drop is at least the viscous dissipation
        assert E1 - E0 <= -P.s * P.gamma * S.edge_dissipation(uh, P.h) + 1e-9
        rho, vel = r1, v1


@pytest.mark.parametrize("kind", ["pfc", "cdft"])
@pytest.mark.parametrize("s", [1e-3, 1.0, 10.0])
def test_energy_stable_for_any_step_dense(kind, s):
    """Unconditional energy stability (Thm 5.1) for large steps, with the
    discrete system solved by dense Newton (no multigrid involved)."""
    n = 6
    rho, vel = _random_state(kind, n, 11)
    if kind == "pfc":
        P, J = pfc_params(1.0, s, alpha=0.6), None
        rho = rho - 0.57
    else:
        P, J = cdft_params((n, n), 1.0, s, 1.0)
    E0 = S.energy(rho, vel, P, J)[0]
    r1, v1, g, nr = newton.solve_dense(rho, vel, P, J=J, tol=1e-11)
    assert nr <= 1e-11
    E1 = S.energy(r1, v1, P, J)[0]
    assert E1 <= E0 + 1e-10
    assert abs(S.mass(r1, P.h) - S.mass(rho, P.h)) < 1e-12


@pytest.mark.parametrize("kind", ["pfc", "cdft"])
def test_fas_matches_dense_newton(kind):
    """The FAS solution equals the dense-Newton solution of N(g) = S."""
    n = 8
    rho, vel = _random_state(kind, n, 3)
    if kind == "pfc":
        P, J = pfc_params(0.5, 0.01), None
    else:
        P, J = cdft_params((n, n), 17.0 / 16, 0.02, 2.362)
    ra, va, _ = S.step(rho, vel, P, S.SolverOpts(tol=1e-13, coarsest=2), J=J)
    rb_, vb, _, _ = newton.solve_dense(rho, vel, P, J=J, tol=1e-14)
    assert np.max(np.abs(ra - rb_)) < 1e-11
    for a, b in zip(va, vb):
        assert np.max(np.abs(a - b)) < 1e-11


def test_lexicographic_and_redblack_reach_the_same_solution():
    """The paper's lexicographic ordering and red-black ordering share the
    fixed point (the discrete solution)."""
    n = 8
    rho, vel = _random_state("pfc", n, 5)
    P = pfc_params(0.5, 0.01)
    a = S.step(rho, vel, P, S.SolverOpts(tol=1e-13, ordering="lex", coarsest=2))
    b = S.step(rho, vel, P, S.SolverOpts(tol=1e-13, ordering="redblack", coarsest=2))
    assert np.max(np.abs(a[0] - b[0])) < 1e-11
    assert np.max(np.abs(a[1][0] - b[1][0])) < 1e-11


def test_3d_invariants():
    """3-D restatement: mass exact, energy non-increasing, uniform fixed point
    and a dense-Newton check on 4^3."""
    n = 8
    rng = np.random.default_rng(9)
    rho = 0.8 + 0.05 * rng.uniform(-1, 1, (n, n, n))
    vel = [0.05 * rng.standard_normal((n, n, n)) for _ in range(3)]
    P = S.Params(kind=S.PFC, dim=3, h=0.9, s=0.02, alpha=0.6)
    E0 = S.energy(rho, vel, P)[0]
    r1, v1, info = S.step(rho, vel, P, S.SolverOpts(tol=1e-12, coarsest=2))
    assert abs(S.mass(r1, P.h) - S.mass(rho, P.h)) < 1e-12
    assert S.energy(r1, v1, P)[0] <= E0
    m = 4
    rho4, vel4 = rho[:m, :m, :m].copy(), [x[:m, :m, :m].copy() for x in vel]
    ra, va, _ = S.step(rho4, vel4, P, S.SolverOpts(tol=1e-13, coarsest=2))
    rb_, vb, _, _ = newton.solve_dense(rho4, vel4, P, tol=1e-14)
    assert np.max(np.abs(ra - rb_)) < 1e-11
    u = np.full((n, n, n), 0.8)
    z = [np.zeros_like(u)] * 3
    r2, v2, info = S.step(u, z, P, S.SolverOpts(tol=1e-12))
    assert info["cycles"] == 0 and np.array_equal(r2, u)


def test_refinement_order_pfc():
    """Sec. 6.1: along s = 0.025 h^2 the Cauchy errors rho^h - rho^{h/2}[2i,2j]
    fall at second order.  Soft pin on the 32/64/128 rungs of the PFC test
    (t = 0.1), where the observed rate approaches 2 from below: rate in
    [1.4, 3] for rho and u."""
    T = 0.1
    sols = {}
    for n in (32, 64, 128):
        rho, h = inputs.smooth_convergence_field(n, kind="pfc")
        vel = [np.zeros((n, n)), np.zeros((n, n))]
        s = 0.025 * h * h
        P = pfc_params(h, s, alpha=0.975, w_damp=0.0)
        # the weighted residual floor of the PFC rows grows like h^-4
        opts = S.SolverOpts(tol=1e-12 if n <= 64 else 1e-10)
        for _ in range(int(round(T / s))):
            rho, vel, _ = S.step(rho, vel, P, opts)
        sols[n] = (rho, vel[0])
    for c in (0, 1):
        e1 = np.sqrt(np.mean((sols[32][c] - sols[64][c][::2, ::2]) ** 2))
        e2 = np.sqrt(np.mean((sols[64][c] - sols[128][c][::2, ::2]) ** 2))
        rate = math.log2(e1 / e2)
        assert 1.4 <= rate <= 3.0, (c, e1, e2, rate)
