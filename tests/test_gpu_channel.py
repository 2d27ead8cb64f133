"""The 2-D PFC channel (walls in y: App. E.2 ghost rules, moving walls of
Sec. 6.3) through the C ABI against the channel oracle, element by element
on the same seeded inputs.  Tolerances as for the periodic path: float64
1e-10, mixed 1e-8 relative per field, both solvers converged to the same
float64 residual; the GPU runs the oracle's hierarchy (coarsest 4, 20
coarse sweeps)."""
import numpy as np
import pytest

from oracle import channel as Ch
from oracle import scheme as S
from paper_1503_07416_gb300 import fm
from tests.helpers import assert_parity, maxrel

pytestmark = pytest.mark.gpu

TOL = {fm.FM_FP64: 1e-10, fm.FM_MIXED: 1e-8}
H = 0.9


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1503_07416_gb300 import build
    build.build_library()
    fm.lib()


def _state(shape, seed, amp_u=0.03):
    rng = np.random.default_rng(seed)
    rho = 0.8 + 0.05 * rng.uniform(-1, 1, shape)
    vel = [amp_u * rng.standard_normal(shape) for _ in range(2)]
    return rho, vel


def _params(s=0.02, sigma=1.0):
    return S.Params(kind=S.PFC, dim=2, h=H, s=s, alpha=0.6, w_damp=0.0, sigma=sigma)


def _solver(shape, precision, walls, tol=1e-12, **kw):
    ny, nx = shape
    return fm.Solver("pfc", (nx, ny), H, alpha=0.6, precision=precision, tol=tol, w_damp=0.0, max_cycles=80,
                     walls=fm.FM_WALLS_Y, u_wall=walls, coarsest=4, ncoarse=20, **kw)


@pytest.mark.parametrize("walls", [(0.0, 0.0), (-0.1, 0.15)])
@pytest.mark.parametrize("precision", [fm.FM_FP64, fm.FM_MIXED])
def test_channel_steps_match_oracle(precision, walls):
    """96 x 64 channel (x periodic, 96 points; 64 rows between the walls),
    walls at rest and moving, two steps each against the oracle's."""
    shape = (64, 96)
    rho, vel = _state(shape, 5)
    P = _params()
    W = Ch.Walls(*walls)
    sol = _solver(shape, precision, walls)
    for step in range(2):
        sol.set_fields(rho, vel)
        info = sol.step(P.s)
        rg, vg = sol.get_fields()
        ro, vo, oinfo = Ch.step(rho, vel, P, W, S.SolverOpts(tol=1e-12))
        assert info.res <= 1e-12
        assert_parity(rg, vg, ro, vo, TOL[precision], (step, info.cycles, oinfo["cycles"]))
        rho, vel = ro, vo
    sol.close()


def test_couette_flow_is_a_fixed_point_on_the_gpu():
    """Plane Couette flow between walls at -U and +U with uniform density:
    zero V-cycles, the state returned unchanged to round-off."""
    ny, nx, U = 32, 32, 0.2
    y = (np.arange(ny) + 0.5) * H
    u = (-U + 2 * U * y / (ny * H))[:, None] * np.ones((ny, nx))
    rho = np.full((ny, nx), 0.8)
    vel = [u, np.zeros((ny, nx))]
    sol = _solver((ny, nx), fm.FM_FP64, (-U, U))
    sol.set_fields(rho, vel)
    info = sol.step(0.02)
    rg, vg = sol.get_fields()
    assert info.cycles == 0 and info.res0 < 1e-13
    assert np.max(np.abs(rg - rho)) < 1e-14 and np.max(np.abs(vg[0] - u)) < 1e-14 and np.max(np.abs(vg[1])) < 1e-14
    sol.close()


@pytest.mark.parametrize("precision", [fm.FM_FP64, fm.FM_MIXED])
def test_channel_mass_and_energy_walls_at_rest(precision):
    """Thm 5.1 with walls at rest on the device: mass to round-off and the
    energy non-increasing over 20 steps (128 x 64)."""
    shape = (64, 128)
    rho, vel = _state(shape, 9)
    sol = _solver(shape, precision, (0.0, 0.0), tol=1e-10)
    sol.set_fields(rho, vel)
    M0 = sol.mass()
    E0 = sol.energy()[0]
    for _ in range(20):
        sol.step(0.02)
        assert abs(sol.mass() - M0) <= 1e-13 * abs(M0)
        E = sol.energy()[0]
        assert E <= E0 + 1e-9
        E0 = E
    P = _params()
    rg, vg = sol.get_fields()
    assert abs(sol.energy()[0] - Ch.energy(rg, vg, P)[0]) <= 1e-12 * abs(E0)
    sol.close()


def test_channel_prepare_and_residual_rows():
    """omega^k, S and g^0 after fm_prepare, and r = S - N(g) of an arbitrary g,
    against the oracle, with moving walls."""
    shape = (32, 48)
    rho, vel = _state(shape, 13, amp_u=0.1)
    P = _params(s=0.03)
    W = Ch.Walls(-0.2, 0.1)
    sol = _solver(shape, fm.FM_FP64, (W.u_bot, W.u_top))
    sol.set_fields(rho, vel)
    fm.fm_prepare(sol.handle, P.s)
    om = Ch.vorticity(vel, H, W)
    Sx = Ch.source(rho, vel, om, P, W)
    g0 = Ch.initial_iterate(rho, vel, P, W)
    assert maxrel(sol.aux(fm.FM_AUX_OMEGA, 0), om[0]) < 1e-13
    for c in range(5):
        assert maxrel(sol.aux(fm.FM_AUX_SOURCE, c), Sx[c]) < 1e-13, c
        assert maxrel(sol.aux(fm.FM_AUX_ITERATE, c), g0[c]) < 1e-13, c
    rng = np.random.default_rng(3)
    g = [x + 0.01 * rng.standard_normal(shape) for x in g0]
    r = [np.empty(shape) for _ in g]
    nrm = fm.fm_residual(sol.handle, g, r)
    ro = Ch.residual(g, Sx, Ch.Coeffs(rho, om), P, W)
    for a, b in zip(r, ro):
        assert np.max(np.abs(a - b)) <= 1e-12 * max(1.0, np.max(np.abs(b)))
    assert abs(nrm - S.res_norm(ro, H)) <= 1e-12 * S.res_norm(ro, H)
    sol.close()


@pytest.mark.parametrize("precision", [fm.FM_FP64, fm.FM_MIXED])
def test_channel_graph_and_launch_by_launch_agree_bitwise(precision):
    shape = (64, 64)
    rho, vel = _state(shape, 21)
    out = []
    for profile in (False, True):
        sol = _solver(shape, precision, (-0.05, 0.05))
        fm.fm_profile(sol.handle, profile)
        sol.set_fields(rho, vel)
        cyc = [sol.step(0.02).cycles for _ in range(2)]
        out.append((sol.get_fields(), cyc))
        sol.close()
    (ra, va), ca = out[0]
    (rb, vb), cb = out[1]
    assert ca == cb and np.array_equal(ra, rb) and all(np.array_equal(a, b) for a, b in zip(va, vb))


def test_channel_rejects_what_it_does_not_support():
    with pytest.raises(fm.FMError):  # CDFT: no wall form of the convolution
        fm.Solver("cdft", (32, 32), 0.5, nu=2.362, walls=fm.FM_WALLS_Y)
    with pytest.raises(fm.FMError):  # 3-D
        fm.Solver("pfc", (16, 16, 16), 0.9, dim=3, alpha=0.6, walls=fm.FM_WALLS_Y)
    with pytest.raises(fm.FMError):
        fm.Batch("pfc", [32, 32], 0.9, alpha=0.6, walls=fm.FM_WALLS_Y)
    sol = _solver((32, 32), fm.FM_FP64, (0.0, 0.0))
    rho, vel = _state((32, 32), 1)
    sol.set_fields(rho, vel)
    fm.fm_prepare(sol.handle, 0.02)
    e = [np.zeros((32, 32)) for _ in range(5)]
    with pytest.raises(fm.FMError):
        fm.fm_smooth(sol.handle, e, e, 1)
    sol.close()
