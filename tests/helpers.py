"""Test helpers: build the oracle's parameters and the CUDA solver from one
workload description, and compare fields."""
import numpy as np

from oracle import scheme as S


def oracle_setup(rho, prm, w_damp=None, tol=None):
    kind = S.PFC if prm["kind"] == "pfc" else S.CDFT
    J = None
    ce = 0.0
    if kind == S.CDFT:
        J, ce = S.cdft_setup(rho.shape, prm["h"], prm["nu"])
    P = S.Params(kind=kind, dim=prm["dim"], h=prm["h"], s=prm["dt"], gamma=prm.get("gamma", 2.0),
                 alpha=prm.get("alpha", 0.0), ce=ce, delta=prm.get("delta", 0.0),
                 w_damp=prm.get("w_damp", 0.5) if w_damp is None else w_damp)
    opts = S.SolverOpts(tol=prm.get("tol", 1e-10) if tol is None else tol, max_cycles=80)
    return P, opts, J


def gpu_solver(rho, prm, precision=0, w_damp=None, tol=None, **kw):
    from paper_1503_07416_gb300 import fm
    n = list(reversed(rho.shape))
    params = dict(tol=prm.get("tol", 1e-10) if tol is None else tol,
                  w_damp=prm.get("w_damp", 0.5) if w_damp is None else w_damp,
                  delta=prm.get("delta", 0.0), gamma=prm.get("gamma", 2.0), max_cycles=80)
    params.update(kw)
    return fm.Solver(prm["kind"], n, prm["h"], dim=prm["dim"], alpha=prm.get("alpha", 0.0),
                     nu=prm.get("nu", 0.0), precision=precision, **params)


def rel(a, b):
    """||a - b||_2 / ||b||_2 (absolute when b vanishes)."""
    nb = float(np.linalg.norm(b))
    d = float(np.linalg.norm(a - b))
    return d / nb if nb > 0 else d


def maxrel(a, b):
    """max |a - b| / max |b| (absolute when b vanishes): the element-wise
    bound, which a single wrong point cannot hide under a whole-field norm."""
    mb = float(np.max(np.abs(b)))
    d = float(np.max(np.abs(a - b)))
    return d / mb if mb > 0 else d


def field_errors(rg, vg, ro, vo):
    """Per field (rho, then each velocity component): (2-norm relative error,
    element-wise relative error) of the GPU fields against the oracle's."""
    pairs = [(rg, ro)] + list(zip(vg, vo))
    return [(rel(a, b), maxrel(a, b)) for a, b in pairs]


def assert_parity(rg, vg, ro, vo, bound, ctx=None):
    """Both bounds per field: ||a - b||_2 <= bound ||b||_2 and
    max |a - b| <= bound max |b|."""
    errs = field_errors(rg, vg, ro, vo)
    worst = max(max(e) for e in errs)
    assert worst <= bound, (ctx, errs)
    return worst
