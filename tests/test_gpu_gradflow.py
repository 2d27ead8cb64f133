"""The gradient-flow model (Sec. 3, Thm 3.3, Eq. gradient_scheme) through the
C ABI against the gradient-flow oracle, element by element on the same
seeded inputs.  Tolerances as for the hydrodynamic path: float64 path
1e-10, mixed path (float32 cycle inside the float64 residual loop) 1e-8,
relative per field, both solvers converged to the same float64 residual;
the paper's damping w = 0.5 on both sides."""
import math

import numpy as np
import pytest

from oracle import gradflow as G
from oracle import scheme as S
from paper_1503_07416_gb300 import fm
from tests.helpers import maxrel, rel

pytestmark = pytest.mark.gpu

TOL = {fm.FM_FP64: 1e-10, fm.FM_MIXED: 1e-8}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1503_07416_gb300 import build
    build.build_library()
    fm.lib()


def _case(kind, n, dim=2, seed=3):
    rng = np.random.default_rng(seed)
    shape = (n,) * dim
    if kind == "pfc":
        rho = 0.8 + 0.05 * rng.uniform(-1, 1, shape)
        prm = dict(h=0.9, s=0.05, alpha=0.6)
    else:
        rho = 0.1 * math.pi * (1 + 0.1 * rng.uniform(0, 1, shape))
        prm = dict(h=17.0 / 32, s=0.05, nu=2.362)
    return rho, prm


def _oracle_params(kind, rho, prm):
    if kind == "pfc":
        return S.Params(kind=S.PFC, dim=rho.ndim, h=prm["h"], s=prm["s"], alpha=prm["alpha"], w_damp=0.5), None
    J, ce = S.cdft_setup(rho.shape, prm["h"], prm["nu"])
    return S.Params(kind=S.CDFT, dim=rho.ndim, h=prm["h"], s=prm["s"], ce=ce, delta=1e-10, w_damp=0.5), J


def _solver(kind, rho, prm, precision, tol, **kw):
    n = list(reversed(rho.shape))
    extra = dict(alpha=prm["alpha"]) if kind == "pfc" else dict(nu=prm["nu"], delta=1e-10)
    # the oracle's hierarchy (down to 4 points a side, 20 sweeps on the coarsest grid)
    mg = dict(coarsest=4, ncoarse=20)
    mg.update(kw)
    return fm.Solver(kind, n, prm["h"], dim=rho.ndim, precision=precision, tol=tol, w_damp=0.5,
                     model=fm.FM_GRADFLOW, max_cycles=100, **extra, **mg)


@pytest.mark.parametrize("precision", [fm.FM_FP64, fm.FM_MIXED])
@pytest.mark.parametrize("kind,n,dim", [("pfc", 64, 2), ("cdft", 64, 2), ("pfc", 96, 2), ("pfc", 16, 3),
                                        ("cdft", 16, 3)])
def test_gradflow_steps_match_oracle(kind, n, dim, precision):
    """Three steps (96^2: a grid whose levels 96 -> 48 -> 24 stop at an even
    size; 16^3: a single 3-D level), each against the oracle's step of the
    same state, with mass to round-off and F non-increasing."""
    rho, prm = _case(kind, n, dim)
    P, J = _oracle_params(kind, rho, prm)
    tol = 1e-12
    sol = _solver(kind, rho, prm, precision, tol)
    M0 = sol_mass = None
    for step in range(3):
        sol.set_fields(rho, None)
        if M0 is None:
            M0 = sol.mass()
        F0 = sol.energy()[1]
        info = sol.step(prm["s"])
        rg, _ = sol.get_fields()
        ro, oinfo = G.step(rho, P, S.SolverOpts(tol=tol, max_cycles=100), J=J)
        assert info.res <= tol
        err = max(rel(rg, ro), maxrel(rg, ro))
        assert err <= TOL[precision], (step, err, info.cycles, oinfo["cycles"])
        sol_mass = sol.mass()
        assert abs(sol_mass - M0) <= 1e-13 * abs(M0)
        assert sol.energy()[1] <= F0 + 1e-10 * max(1.0, abs(F0))
        rho = ro
    sol.close()


@pytest.mark.parametrize("kind", ["pfc", "cdft"])
def test_gradflow_prepare_and_residual_rows(kind):
    """S and g^0 after fm_prepare, and r = S - N(g) for an arbitrary g, against
    the oracle's source, initial iterate and residual."""
    rho, prm = _case(kind, 32, 2, seed=7)
    P, J = _oracle_params(kind, rho, prm)
    sol = _solver(kind, rho, prm, fm.FM_FP64, 1e-12)
    sol.set_fields(rho, None)
    fm.fm_prepare(sol.handle, prm["s"])
    C = S.conv_fft(J, rho, P.h) if kind == "cdft" else None
    Sx = G.source(rho, P, C)
    g0 = G.initial_iterate(rho, P)
    for c in range(len(Sx)):
        assert maxrel(sol.aux(fm.FM_AUX_SOURCE, c), Sx[c]) < 1e-13, c
        assert maxrel(sol.aux(fm.FM_AUX_ITERATE, c), g0[c]) < 1e-13, c
    rng = np.random.default_rng(17)
    g = [rho + 0.01 * rng.standard_normal(rho.shape)]
    if kind == "pfc":
        g += [rng.standard_normal(rho.shape), rng.standard_normal(rho.shape)]
    r = [np.empty_like(rho) for _ in g]
    nrm = fm.fm_residual(sol.handle, g, r)
    ro = G.residual(g, Sx, P)
    for a, b in zip(r, ro):
        assert np.max(np.abs(a - b)) <= 1e-12 * max(1.0, np.max(np.abs(b)))
    assert abs(nrm - S.res_norm(ro, P.h)) <= 1e-12 * S.res_norm(ro, P.h)
    sol.close()


@pytest.mark.parametrize("precision", [fm.FM_FP64, fm.FM_MIXED])
def test_gradflow_large_grid_and_graph_modes(precision, monkeypatch):
    """A 512^2 PFC gradient-flow step (several waves of every kernel) against
    the oracle, and the graph and launch-by-launch modes bit for bit."""
    rho, prm = _case("pfc", 512, 2, seed=5)
    P, J = _oracle_params("pfc", rho, prm)
    tol = 1e-11
    ro, _ = G.step(rho, P, S.SolverOpts(tol=tol, max_cycles=100), J=J)
    out = []
    for profile in (False, True):
        sol = _solver("pfc", rho, prm, precision, tol)
        fm.fm_profile(sol.handle, profile)
        sol.set_fields(rho, None)
        info = sol.step(prm["s"])
        rg, vg = sol.get_fields()
        sol.close()
        assert info.res <= tol
        assert max(rel(rg, ro), maxrel(rg, ro)) <= TOL[precision]
        assert all(np.all(v == 0) for v in vg)
        out.append((rg, info.cycles))
    assert out[0][1] == out[1][1] and np.array_equal(out[0][0], out[1][0])


def test_gradflow_rejects_hydrodynamic_only_calls():
    rho, prm = _case("pfc", 32, 2)
    sol = _solver("pfc", rho, prm, fm.FM_FP64, 1e-12)
    sol.set_fields(rho, None)
    fm.fm_prepare(sol.handle, prm["s"])
    e = [np.zeros_like(rho) for _ in range(3)]
    with pytest.raises(fm.FMError):
        fm.fm_smooth(sol.handle, e, e, 1)
    sol.close()
    with pytest.raises(fm.FMError):
        fm.Batch("pfc", [32, 32], 0.9, alpha=0.6, model=fm.FM_GRADFLOW)
