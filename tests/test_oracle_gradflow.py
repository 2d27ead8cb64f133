"""Pins of the gradient-flow oracle (Sec. 3, Thm 3.3, Eq. gradient_scheme)
against what the paper and the mathematics fix: exact mass, the energy
decay bound of Thm 3.3 with its dissipation term, the closed-form
amplification of a small Fourier mode, the uniform fixed point, and FAS
equal to a dense Newton solve (no multigrid) on tiny grids.  The smoother
runs with the paper's damping w = 0.5 (App. G.3): undamped red-black point
sweeps of the sixth-order PFC flow do not converge."""
import math

import numpy as np
import pytest

from oracle import gradflow as G
from oracle import scheme as S


def pfc_params(h, s, alpha=0.6, **kw):
    return S.Params(kind=S.PFC, dim=2, h=h, s=s, alpha=alpha, w_damp=0.5, **kw)


def cdft_params(shape, h, s, nu=2.362, **kw):
    J, ce = S.cdft_setup(shape, h, nu)
    return S.Params(kind=S.CDFT, dim=2, h=h, s=s, ce=ce, delta=1e-10, w_damp=0.5, **kw), J


def _state(kind, n, seed, dim=2):
    rng = np.random.default_rng(seed)
    shape = (n,) * dim
    if kind == "pfc":
        return 0.8 + 0.05 * rng.uniform(-1, 1, shape)
    return 0.1 * math.pi * (1 + 0.1 * rng.uniform(0, 1, shape))


@pytest.mark.parametrize("kind", ["pfc", "cdft"])
def test_mass_and_thm33_energy_bound(kind):
    """Thm 3.3: (rho^{k+1} || 1) = (rho^k || 1) and, through the convex
    splitting inequality and summation by parts,
    F^{k+1} - F^k <= -s ||grad_h mu^{k+1}||^2 (edge norms) <= 0."""
    n = 32
    rho = _state(kind, n, 3)
    if kind == "pfc":
        P, J = pfc_params(0.9, 0.05), None
    else:
        P, J = cdft_params((n, n), 17.0 / 32, 0.05)
    M0 = S.mass(rho, P.h)
    for _ in range(4):
        F0 = G.free_energy(rho, P, J)
        r1, info = G.step(rho, P, S.SolverOpts(tol=1e-12), J=J)
        F1 = G.free_energy(r1, P, J)
        assert abs(S.mass(r1, P.h) - M0) <= 1e-13 * abs(M0)
        diss = P.s * G.edge_norm(info["mu"], P.h)
        assert diss > 0
        assert F1 - F0 <= -diss + 1e-10 * max(1.0, abs(F0)), (F1 - F0, diss)
        rho = r1


@pytest.mark.parametrize("kind", ["pfc", "cdft"])
@pytest.mark.parametrize("s", [1e-2, 1.0, 10.0])
def test_energy_stable_for_any_step_dense(kind, s):
    """Unconditional stability (any s > 0) with the discrete system solved by
    dense Newton, so no multigrid is involved."""
    n = 6
    rho = _state(kind, n, 11)
    if kind == "pfc":
        P, J = pfc_params(1.0, s), None
    else:
        P, J = cdft_params((n, n), 1.0, s, nu=1.0)
    r1, g, nr = G.solve_dense(rho, P, J=J, tol=1e-11)
    assert nr <= 1e-11
    assert G.free_energy(r1, P, J) <= G.free_energy(rho, P, J) + 1e-10
    assert abs(S.mass(r1, P.h) - S.mass(rho, P.h)) < 1e-12


@pytest.mark.parametrize("kind", ["pfc", "cdft"])
@pytest.mark.parametrize("axis", [0, 1])
def test_linearised_single_mode_step(kind, axis):
    """rho^k = rho_bar + a cos(k.x) with a small: the linearised scheme gives
    A = a (1 + s lam c0) / (1 - s lam c1), lam = -(4/h^2) sin^2(kh/2) the
    symbol of Lap_h, c1 = dF_c'' (PFC: psi_bar^2 + alpha + lam^2; CDFT:
    1/rho_bar + 2 c_e) and c0 the explicit part (PFC: 2 lam; CDFT:
    -(2 c_e + Jhat(k)))."""
    n = 32
    if kind == "pfc":
        h, s, rb = 0.9, 0.5, 0.8
        P, J = pfc_params(h, s), None
    else:
        h, s, rb = 17.0 / 32, 0.5, 0.1 * math.pi
        P, J = cdft_params((n, n), h, s)
    x = np.arange(n) * h
    X, Y = np.meshgrid(x, x, indexing="xy")
    Z = X if axis == 0 else Y
    k = 2 * math.pi * 3 / (n * h)
    a = 1e-6
    rho = rb + a * np.cos(k * Z)
    lam = -4.0 / h ** 2 * math.sin(k * h / 2) ** 2
    if kind == "pfc":
        psi = rb - 1.5
        c1, c0 = psi * psi + P.alpha + lam * lam, 2 * lam
    else:
        jhat = float(np.sum(J * np.cos(k * X))) * h * h
        c1, c0 = 1.0 / rb + 2 * P.ce, -(2 * P.ce + jhat)
    A = a * (1 + s * lam * c0) / (1 - s * lam * c1)
    r1, _ = G.step(rho, P, S.SolverOpts(tol=1e-12, max_cycles=80), J=J)
    got = 2 * np.mean((r1 - rb) * np.cos(k * Z))
    assert abs(got - A) < 1e-5 * abs(a), (got, A)


@pytest.mark.parametrize("kind", ["pfc", "cdft"])
def test_uniform_state_is_a_fixed_point(kind):
    n = 16
    if kind == "pfc":
        P, J, rb = pfc_params(0.9, 0.05), None, 0.8
    else:
        (P, J), rb = cdft_params((n, n), 17.0 / 16, 0.05), 0.1 * math.pi
    rho = np.full((n, n), rb)
    r1, info = G.step(rho, P, S.SolverOpts(tol=1e-12), J=J)
    assert info["cycles"] == 0 and np.array_equal(r1, rho)


@pytest.mark.parametrize("kind", ["pfc", "cdft"])
def test_fas_matches_dense_newton(kind):
    n = 8
    rho = _state(kind, n, 5)
    if kind == "pfc":
        P, J = pfc_params(0.9, 0.1), None
    else:
        P, J = cdft_params((n, n), 17.0 / 16, 0.1)
    ra, _ = G.step(rho, P, S.SolverOpts(tol=1e-13, coarsest=2), J=J)
    rb_, _, _ = G.solve_dense(rho, P, J=J, tol=1e-14)
    assert np.max(np.abs(ra - rb_)) < 1e-11


def test_3d_mass_energy_and_dense_newton():
    """3-D (7-point Laplacian): mass exact, Thm 3.3 bound, FAS = dense Newton
    on 4^3."""
    n = 8
    rho = _state("pfc", n, 9, dim=3)
    P = S.Params(kind=S.PFC, dim=3, h=0.9, s=0.05, alpha=0.6, w_damp=0.5)
    F0 = G.free_energy(rho, P)
    r1, info = G.step(rho, P, S.SolverOpts(tol=1e-12, coarsest=2))
    assert abs(S.mass(r1, P.h) - S.mass(rho, P.h)) < 1e-12
    assert G.free_energy(r1, P) - F0 <= -P.s * G.edge_norm(info["mu"], P.h) + 1e-10
    r4 = rho[:4, :4, :4].copy()
    ra, _ = G.step(r4, P, S.SolverOpts(tol=1e-13, coarsest=2))
    rb_, _, _ = G.solve_dense(r4, P, tol=1e-14)
    assert np.max(np.abs(ra - rb_)) < 1e-11
