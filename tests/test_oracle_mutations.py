"""Plant plausible mistakes in the oracle (CPU only) and check that the pins
catch each one.  This shows that the pins are not checking the oracle against
itself: a dropped term, a wrong sign, a wrong index or a wrong weight fails at
least one of them."""
import math

import numpy as np
import pytest

from oracle import scheme as S
import tests.test_oracle_pins as pins


def _garbled_lap(a, h):
    # App. E prints phi_{i-1,j} twice where phi_{i,j-1} is meant
    if a.ndim != 2:
        return _orig["lap"](a, h)
    return (S.sh(a, 0, 1) + S.sh(a, 1, 1) + 2 * S.sh(a, 0, -1) - 4 * a) / (h * h)


def _flipped_cross(om, U):
    return [-x for x in _orig["omega_cross"](om, U)]


def _flipped_cross_3d(om, U):
    # the consistent 3-D analogue of sigma = -1: only the 3-D branch negated
    out = _orig["omega_cross"](om, U)
    return [-x for x in out] if len(U) == 3 else out


def _swapped_cross_3d(om, U):
    # one slot of the 3-D cross product with its operands exchanged
    out = _orig["omega_cross"](om, U)
    if len(U) == 3:
        out[1] = om[0] * U[2] - om[2] * U[0]
    return out


def _curl_x_flipped(vel, h):
    # the x-component of the 3-D centred curl with the wrong sign
    out = _orig["vorticity"](vel, h)
    if len(vel) == 3:
        out[0] = -out[0]
    return out


def _forward_div(F, h):
    return sum((S.sh(F[d], d, 1) - F[d]) / h for d in range(len(F)))


def _inject_only(r):
    return S.inject(r)


def _quartic_wrong(rho, h, alpha):
    t = _orig["pfc_energy_terms"](rho, h, alpha)
    return (3.0 * t[0],) + tuple(t[1:])


def _closure_no_half(g, rk, uk, P):
    return rk - P.s * S.div0([rk * g[1 + a] for a in range(P.dim)], P.h)


def _ce_unweighted(shape, h, nu):
    J, ce = _orig["cdft_setup"](shape, h, nu)
    return J, ce / h ** len(shape)


_orig = {k: getattr(S, k) for k in ("lap", "omega_cross", "div0", "restrict_fw",
                                    "pfc_energy_terms", "closure", "cdft_setup", "vorticity")}


def _all_3d_shears():
    for a, b in pins.SHEAR_3D:
        pins.test_3d_shear_flow_generates_no_cross_flow(a, b)


MUTATIONS = [
    ("lap", _garbled_lap, [lambda: pins.test_stencil_symbols()]),
    ("omega_cross", _flipped_cross, [pins.test_shear_flow_generates_no_cross_flow]),
    ("div0", _forward_div, [lambda: pins.test_linearised_single_mode_step("pfc", 0)]),
    ("restrict_fw", _inject_only, [pins.test_transfers]),
    ("pfc_energy_terms", _quartic_wrong, [pins.test_pfc_energy_of_a_mode]),
    ("closure", _closure_no_half, [lambda: pins.test_mass_energy_and_kinetic_identity("pfc")]),
    ("cdft_setup", _ce_unweighted, [pins.test_ce_closed_form]),
    ("omega_cross", _flipped_cross_3d, [_all_3d_shears]),
    ("omega_cross", _swapped_cross_3d, [_all_3d_shears]),
    ("vorticity", _curl_x_flipped, [_all_3d_shears]),
]

IDS = ["lap", "omega_cross", "div0", "restrict_fw", "pfc_energy_terms", "closure", "cdft_setup",
       "omega_cross_3d_negated", "omega_cross_3d_slot_swapped", "curl_3d_x_negated"]


@pytest.mark.parametrize("name,fn,checks", MUTATIONS, ids=IDS)
def test_pins_catch_planted_mistake(monkeypatch, name, fn, checks):
    monkeypatch.setattr(S, name, fn)
    caught = 0
    for chk in checks:
        try:
            chk()
        except (AssertionError, S.NoConvergence, np.linalg.LinAlgError, FloatingPointError):
            caught += 1
    assert caught == len(checks), f"planted mistake in {name} not caught"


# ---------------------------------------------------------------- gradient flow
from oracle import gradflow as G  # noqa: E402
import tests.test_oracle_gradflow as gpins  # noqa: E402

_gorig = {k: getattr(G, k) for k in ("explicit_mu", "closure", "apply_N")}


def _explicit_sign(rk, P, C=None):
    return -_gorig["explicit_mu"](rk, P, C)


def _closure_minus(g, rk, P, Emu=None):
    rho = rk - P.s * S.lap(G.mu_of(g, P, Emu), P.h)
    return np.sqrt(rho * rho + P.delta * P.delta)


def _cubic_unscaled(g, P):
    out = _gorig["apply_N"](g, P)
    if P.kind == S.PFC:
        psi = g[0] - 1.5
        out[1] = out[1] - (2.0 / 3.0) * psi ** 3
    return out


def _gf_modes():
    for kind in ("pfc", "cdft"):
        gpins.test_linearised_single_mode_step(kind, 0)


G_MUTATIONS = [
    ("explicit_mu", _explicit_sign, [_gf_modes]),
    ("closure", _closure_minus, [_gf_modes, lambda: gpins.test_mass_and_thm33_energy_bound("pfc")]),
    ("apply_N", _cubic_unscaled, [lambda: gpins.test_linearised_single_mode_step("pfc", 1)]),
]


@pytest.mark.parametrize("name,fn,checks", G_MUTATIONS, ids=["gf_explicit_sign", "gf_closure_sign",
                                                             "gf_cubic_weight"])
def test_gradflow_pins_catch_planted_mistake(monkeypatch, name, fn, checks):
    monkeypatch.setattr(G, name, fn)
    caught = 0
    for chk in checks:
        try:
            chk()
        except (AssertionError, S.NoConvergence, np.linalg.LinAlgError, FloatingPointError):
            caught += 1
    assert caught == len(checks), f"planted mistake in gradflow.{name} not caught"


# ---------------------------------------------------------------- channel walls
from oracle import channel as Ch  # noqa: E402
import tests.test_oracle_channel as cpins  # noqa: E402

_corig = {"ghost": Ch.ghost}


def _normal_even(row, typ, U):
    return row if typ == Ch.VN else _corig["ghost"](row, typ, U)


def _wall_speed_once(row, typ, U):
    return U - row if typ == Ch.UT else _corig["ghost"](row, typ, U)


def _scalar_dirichlet(row, typ, U):
    return 0.0 * row if typ == Ch.SCAL else _corig["ghost"](row, typ, U)


C_MUTATIONS = [
    ("normal_velocity_even", _normal_even, [cpins.test_mass_energy_and_kinetic_identity_walls_at_rest]),
    ("wall_speed_not_doubled", _wall_speed_once, [cpins.test_couette_flow_is_an_exact_fixed_point]),
    ("scalar_ghost_zero", _scalar_dirichlet, [cpins.test_uniform_state_is_a_fixed_point]),
]


@pytest.mark.parametrize("label,fn,checks", C_MUTATIONS, ids=[m[0] for m in C_MUTATIONS])
def test_channel_pins_catch_planted_mistake(monkeypatch, label, fn, checks):
    monkeypatch.setattr(Ch, "ghost", fn)
    caught = 0
    for chk in checks:
        try:
            with np.errstate(all="ignore"):
                chk()
        except (AssertionError, S.NoConvergence, np.linalg.LinAlgError, FloatingPointError):
            caught += 1
    assert caught == len(checks), f"planted mistake {label} not caught"
