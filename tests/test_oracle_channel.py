"""Pins of the channel oracle (walls in y: App. E.2 ghost rules, moving
walls of Sec. 6.3) against what the paper and the mathematics fix: mass
conservation and unconditional energy stability with walls at rest (Thm 5.1
carried over by App. E.2), the exact kinetic-energy identity with the wall
edges, plane Couette flow between moving walls as an exact fixed point (and
not a fixed point with the App. G vorticity sign), the closed-form
amplification of a wall eigenmode, the uniform fixed point, and FAS equal to
dense Newton."""
import math

import numpy as np
import pytest

from oracle import channel as Ch
from oracle import scheme as S


def params(h=0.9, s=0.02, alpha=0.6, **kw):
    kw.setdefault("w_damp", 0.0)
    return S.Params(kind=S.PFC, dim=2, h=h, s=s, alpha=alpha, **kw)


def _state(shape, seed, amp_u=0.03):
    rng = np.random.default_rng(seed)
    rho = 0.8 + 0.05 * rng.uniform(-1, 1, shape)
    vel = [amp_u * rng.standard_normal(shape) for _ in range(2)]
    return rho, vel


def test_mass_energy_and_kinetic_identity_walls_at_rest():
    """Thm 5.1 with walls at rest, and the exact identity
    KE^{k+1} - KE^k + (rho^{k+1} - rho^k || mu^{k+1}) + s gamma D = 0, D the
    edge norms of u^{k+1/2} with the wall edges at weight 1/2."""
    rho, vel = _state((32, 48), 3)
    P = params()
    M0 = S.mass(rho, P.h)
    for _ in range(3):
        E0, _, K0 = Ch.energy(rho, vel, P)
        r1, v1, info = Ch.step(rho, vel, P, opts=S.SolverOpts(tol=1e-12))
        E1, _, K1 = Ch.energy(r1, v1, P)
        assert abs(S.mass(r1, P.h) - M0) <= 1e-13 * abs(M0)
        uh = [0.5 * (a + b) for a, b in zip(v1, vel)]
        D = Ch.edge_dissipation(uh, P.h)
        ident = K1 - K0 + S.inner(r1 - rho, info["g"][3], P.h) + P.s * P.gamma * D
        assert abs(ident) < 1e-10 * max(1.0, abs(E0)), ident
        assert E1 - E0 <= -P.s * P.gamma * D + 1e-10
        rho, vel = r1, v1


@pytest.mark.parametrize("s", [1e-2, 1.0, 10.0])
def test_energy_stable_for_any_step_dense(s):
    """Walls at rest, any s, the system solved by dense Newton."""
    rho, vel = _state((4, 6), 11, amp_u=0.05)
    P = params(h=1.0, s=s)
    E0 = Ch.energy(rho, vel, P)[0]
    r1, v1, _, nr = Ch.solve_dense(rho, vel, P, tol=1e-11)
    assert nr <= 1e-11
    assert Ch.energy(r1, v1, P)[0] <= E0 + 1e-10
    assert abs(S.mass(r1, P.h) - S.mass(rho, P.h)) < 1e-12


def _couette(ny, nx, h, U):
    y = (np.arange(ny) + 0.5) * h
    L = ny * h
    u = (-U + 2.0 * U * y / L)[:, None] * np.ones((ny, nx))
    return u


def test_couette_flow_is_an_exact_fixed_point():
    """Uniform density and the linear shear u = U (2y/L - 1), v = 0 between
    walls moving at -U and +U: u.grad u = 0, Lap u = 0 (the ghost rule puts
    the wall speed at the wall), so with the vector-form vorticity sign the
    first residual is zero to round-off and the step returns the state; the
    App. G sign (sigma = -1) leaves a y-momentum imbalance of rho u u' and
    drives a flow."""
    ny, nx, h, U = 16, 16, 0.9, 0.2
    rho = np.full((ny, nx), 0.8)
    vel = [_couette(ny, nx, h, U), np.zeros((ny, nx))]
    W = Ch.Walls(-U, U)
    r1, v1, info = Ch.step(rho, vel, params(), W, S.SolverOpts(tol=1e-12))
    assert info["hist"][0] < 1e-13
    assert info["cycles"] == 0
    assert np.max(np.abs(r1 - rho)) < 1e-14 and np.max(np.abs(v1[0] - vel[0])) < 1e-14
    r2, v2, info2 = Ch.step(rho, vel, params(sigma=-1.0), W, S.SolverOpts(tol=1e-12))
    assert info2["cycles"] > 0 and np.max(np.abs(r2 - rho)) > 1e-6


def test_wall_eigenmode_amplification():
    """rho = rho_bar + a cos(k y), v = b sin(k y), k = m pi / L_y (cell
    centres y = (j + 1/2) h): cos is even and sin odd about each wall, so they
    are eigenfunctions of the Neumann / no-slip Lap_h and D0 maps one to the
    other; one step of the linearised scheme follows the 2x2 closed form of
    the periodic case."""
    from tests.test_oracle_pins import _linear_mode_prediction
    ny, nx, h, s = 32, 16, 0.5, 0.05
    rb, alpha = 1.5 - 0.07 * math.sqrt(3), 0.975
    y = (np.arange(ny) + 0.5) * h
    k = 3 * math.pi / (ny * h)
    a, b = 1e-6, 0.7e-6
    rho = rb + a * np.cos(k * y)[:, None] * np.ones((ny, nx))
    vel = [np.zeros((ny, nx)), b * np.sin(k * y)[:, None] * np.ones((ny, nx))]
    P = params(h=h, s=s, alpha=alpha, w_damp=0.5)  # undamped sweeps diverge at h = 0.5
    # the ghosts continue cos (even) and sin (odd) across both walls, so the
    # wall mode moves as the periodic mode of the same k
    A, B = _linear_mode_prediction("pfc", rb, a, b, k, h, s, P.gamma, alpha=alpha)
    r1, v1, _ = Ch.step(rho, vel, P, opts=S.SolverOpts(tol=1e-13))
    cy = np.cos(k * y)[:, None]
    sy = np.sin(k * y)[:, None]
    got_A = np.sum((r1 - rb) * cy) / np.sum(cy * cy * np.ones((ny, nx)))
    got_B = np.sum(v1[1] * sy) / np.sum(sy * sy * np.ones((ny, nx)))
    assert abs(got_A - A) < 1e-4 * abs(A), (got_A, A)
    assert abs(got_B - B) < 1e-4 * abs(B), (got_B, B)
    assert np.max(np.abs(v1[0])) < 1e-3 * abs(B)


def test_uniform_state_is_a_fixed_point():
    rho = np.full((16, 16), 0.8)
    vel = [np.zeros((16, 16)), np.zeros((16, 16))]
    r1, v1, info = Ch.step(rho, vel, params(), opts=S.SolverOpts(tol=1e-12))
    assert info["cycles"] == 0 and np.array_equal(r1, rho)


@pytest.mark.parametrize("walls", [(0.0, 0.0), (-0.1, 0.15)])
def test_fas_matches_dense_newton(walls):
    rho, vel = _state((8, 8), 5)
    P = params()
    W = Ch.Walls(*walls)
    ra, va, _ = Ch.step(rho, vel, P, W, S.SolverOpts(tol=1e-13, coarsest=2))
    rb_, vb, _, _ = Ch.solve_dense(rho, vel, P, W, tol=1e-14)
    assert np.max(np.abs(ra - rb_)) < 1e-11
    for x, y in zip(va, vb):
        assert np.max(np.abs(x - y)) < 1e-11


def test_transfers():
    """Cell-centred y transfers: restriction and injection keep constants;
    prolongation keeps constants of a scalar correction and R = 2^-2 P^T for
    the scalar type away from the walls' ghost terms (adjointness in x and in
    the interior of y)."""
    rng = np.random.default_rng(2)
    c = np.full((16, 12), 2.5)
    assert np.allclose(Ch.restrict(c), 2.5) and np.allclose(Ch.inject(c), 2.5)
    assert np.allclose(Ch.prolong(np.full((8, 6), 2.5), Ch.SCAL), 2.5)
    E = rng.standard_normal((8, 6))
    fine = Ch.prolong(E, Ch.SCAL)
    # linear in y between cell centres: the mean of the two children is E
    # wherever E varies linearly
    lin = np.arange(8.0)[:, None] * np.ones((1, 6))
    pf = Ch.prolong(lin, Ch.SCAL)
    assert np.allclose(0.5 * (pf[2:-2:2, ::2] + pf[3:-2:2, ::2]), lin[1:-1])
    assert fine.shape == (16, 12)
