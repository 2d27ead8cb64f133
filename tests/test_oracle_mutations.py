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
                                    "pfc_energy_terms", "closure", "cdft_setup")}

MUTATIONS = [
    ("lap", _garbled_lap, [lambda: pins.test_stencil_symbols()]),
    ("omega_cross", _flipped_cross, [pins.test_shear_flow_generates_no_cross_flow]),
    ("div0", _forward_div, [lambda: pins.test_linearised_single_mode_step("pfc", 0)]),
    ("restrict_fw", _inject_only, [pins.test_transfers]),
    ("pfc_energy_terms", _quartic_wrong, [pins.test_pfc_energy_of_a_mode]),
    ("closure", _closure_no_half, [lambda: pins.test_mass_energy_and_kinetic_identity("pfc")]),
    ("cdft_setup", _ce_unweighted, [pins.test_ce_closed_form]),
]


@pytest.mark.parametrize("name,fn,checks", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_pins_catch_planted_mistake(monkeypatch, name, fn, checks):
    monkeypatch.setattr(S, name, fn)
    caught = 0
    for chk in checks:
        try:
            chk()
        except (AssertionError, S.NoConvergence, np.linalg.LinAlgError, FloatingPointError):
            caught += 1
    assert caught == len(checks), f"planted mistake in {name} not caught"
