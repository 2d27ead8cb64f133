"""Smoother row (App. G.1-G.3): red-black point-block Gauss-Seidel sweeps
through fm_smooth, on the coefficient iterate g^0 of a prepared step and a
right-hand side f = S - N(g^0) computed by the oracle, against the oracle's own
red-black sweeps of N(g) = S from g^0 (the correction e and the oracle's
increment g - g^0 solve the same point systems).

CDFT is compared with the oracle directly: its point block is linear in the
point's own unknowns, so both sides solve identical systems.  The PFC point
block differs by design (the oracle linearises the cubic as App. G.2 prints
it, the CUDA update evaluates it exactly), so for PFC every fused tile
variant is compared with the red launch + black launch pair instead.  Sizes
are chosen so that every variant runs its tiles in several waves: a fused
sweep that read a neighbour tile's already updated values would show here.

Tolerances: float64 1e-11 of max |increment| (the increments are O(1e-2),
the fields O(1), so this is a few hundred ulps of the fields); mixed 2e-5
(float32 point solves of a float32-rounded f and coefficients)."""
import numpy as np
import pytest

from oracle import scheme as S
from paper_1503_07416_gb300 import fm
from tests.helpers import gpu_solver, oracle_setup

pytestmark = pytest.mark.gpu

TOL = {fm.FM_FP64: 1e-11, fm.FM_MIXED: 2e-5}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1503_07416_gb300 import build
    build.build_library()
    fm.lib()


def _case(kind, shape, seed):
    rng = np.random.default_rng(seed)
    if kind == "cdft":
        rho = 0.3 + 0.05 * rng.uniform(0, 1, shape)
        prm = dict(kind="cdft", dim=2, h=34.0 / shape[1], dt=0.02, nu=2.362, delta=1e-10)
    else:
        rho = 0.8 + 0.05 * rng.uniform(-1, 1, shape)
        prm = dict(kind="pfc", dim=2, h=0.9, dt=0.02, alpha=0.6)
    vel = [0.05 * rng.standard_normal(shape) for _ in range(2)]
    return rho, vel, prm


def _oracle(rho, vel, prm, w, sweeps):
    """g^0, f = S - N(g^0) and the increment of `sweeps` oracle sweeps."""
    P, _, J = oracle_setup(rho, prm, w_damp=w)
    om = S.vorticity(vel, P.h)
    C = S.conv_fft(J, rho, P.h) if P.kind == S.CDFT else None
    Sx = S.source(rho, vel, om, P, C)
    c = S.Coeffs(rho, om)
    g0 = S.initial_iterate(rho, vel, P)
    f = S.residual(g0, Sx, c, P)
    g = [x.copy() for x in g0]
    for _ in range(sweeps):
        S.smooth(g, Sx, c, P)
    return f, [a - b for a, b in zip(g, g0)]


def _gpu(rho, vel, prm, f, precision, w, sweeps, variant):
    sol = gpu_solver(rho, prm, precision=precision, w_damp=w)
    try:
        sol.set_fields(rho, vel)
        fm.fm_prepare(sol.handle, prm["dt"])
        e = [np.zeros_like(rho) for _ in f]
        fm.fm_smooth(sol.handle, e, [np.ascontiguousarray(x) for x in f], sweeps, variant)
        return e
    finally:
        sol.close()


def _close(a, b, tol):
    for q, (x, y) in enumerate(zip(a, b)):
        scale = float(np.max(np.abs(y)))
        err = float(np.max(np.abs(x - y)))
        assert err <= tol * scale, (q, err, scale)


@pytest.mark.parametrize("w", [0.0, 0.5])
@pytest.mark.parametrize("sweeps", [1, 2, 3])
@pytest.mark.parametrize("precision", [fm.FM_FP64, fm.FM_MIXED])
def test_cdft_sweeps_match_oracle(precision, sweeps, w):
    """As fm_step runs them (fused pairs, an odd last sweep as two launches),
    on a 64 x 32 grid (CDFT sizes are powers of two for the FFT)."""
    rho, vel, prm = _case("cdft", (32, 64), 3)
    f, de = _oracle(rho, vel, prm, w, sweeps)
    e = _gpu(rho, vel, prm, f, precision, w, sweeps, fm.FM_SWEEP_AUTO)
    _close(e, de, TOL[precision])


@pytest.mark.parametrize("precision", [fm.FM_FP64, fm.FM_MIXED])
def test_cdft_two_colour_sweeps_match_oracle(precision):
    rho, vel, prm = _case("cdft", (64, 32), 4)
    f, de = _oracle(rho, vel, prm, 0.5, 2)
    e = _gpu(rho, vel, prm, f, precision, 0.5, 2, fm.FM_SWEEP_TWO_COLOUR)
    _close(e, de, TOL[precision])


@pytest.mark.parametrize("precision", [fm.FM_FP64, fm.FM_MIXED])
def test_cdft_every_fused_variant_matches_oracle_over_many_waves(precision):
    """512 x 1024: 512 to 1024 tiles per sweep, more than the device holds at
    once for every variant."""
    rho, vel, prm = _case("cdft", (512, 1024), 5)
    f, de = _oracle(rho, vel, prm, 0.0, 2)
    for v in range(fm.FM_SWEEP_VARIANTS):
        try:
            e = _gpu(rho, vel, prm, f, precision, 0.0, 2, v)
        except fm.FMError as err:  # variant too large for shared memory
            assert err.code == fm.FM_EINVAL and precision == fm.FM_FP64
            continue
        _close(e, de, TOL[precision])


@pytest.mark.parametrize("precision", [fm.FM_FP64, fm.FM_MIXED])
def test_pfc_every_fused_variant_matches_two_colour_launches(precision):
    """PFC, 1002 x 1000 points (sides not multiples of any tile; rows not a
    whole number of 16-byte chunks, so the tiles are staged element by
    element), 4 sweeps."""
    rho, vel, prm = _case("pfc", (1000, 1002), 6)
    f, _ = _oracle(rho, vel, prm, 0.0, 0)
    ref = _gpu(rho, vel, prm, f, precision, 0.0, 4, fm.FM_SWEEP_TWO_COLOUR)
    tol = 1e-12 if precision == fm.FM_FP64 else 2e-5
    for v in range(fm.FM_SWEEP_VARIANTS):
        try:
            e = _gpu(rho, vel, prm, f, precision, 0.0, 4, v)
        except fm.FMError as err:
            assert err.code == fm.FM_EINVAL and precision == fm.FM_FP64
            continue
        _close(e, ref, tol)


@pytest.mark.parametrize("precision", [fm.FM_FP64, fm.FM_MIXED])
@pytest.mark.parametrize("kind,shape", [("pfc", (1000, 1002)), ("pfc", (18, 10)), ("pfc", (6, 140)),
                                        ("cdft", (64, 128))])
def test_two_sweep_pass_equals_one_sweep_passes(kind, shape, precision, monkeypatch):
    """The two-sweep variants run the same point update on the same values
    as the one-sweep variants with the same blocks -- marching 18..23 against
    12..17, tiles 24..26 against 0, 4, 8, small tiles 31 and 33 against 30
    and 32, the 32 x 14 tiles of 35 against the 32 x 16 ones of 0 -- only in
    another order of
    independent points, so the results agree bit for bit: 2 sweeps (one pass)
    and 5 (two passes and a two-colour sweep), on grids with ragged strips
    and tiles, fewer rows than a block and fewer columns than a strip."""
    monkeypatch.setenv("FM_RB_VARIANT", "0")  # no autotuning at create
    rho, vel, prm = _case(kind, shape, 9)
    f, _ = _oracle(rho, vel, prm, 0.0, 0)
    pairs = [(18 + m, 12 + m) for m in range(6)] + [(24 + k, 4 * k) for k in range(3)] + [(31, 30), (33, 32), (35, 0)]
    for sweeps in (2, 5):
        for v2, v1 in pairs:
            try:
                one = _gpu(rho, vel, prm, f, precision, 0.0, sweeps, v1)
                two = _gpu(rho, vel, prm, f, precision, 0.0, sweeps, v2)
            except fm.FMError as err:
                assert err.code == fm.FM_EINVAL and precision == fm.FM_FP64
                continue
            for q, (a, b) in enumerate(zip(two, one)):
                assert np.array_equal(a, b), (sweeps, v2, q, float(np.max(np.abs(a - b))))


@pytest.mark.parametrize("precision", [fm.FM_FP64, fm.FM_MIXED])
@pytest.mark.parametrize("kind,shape", [("pfc", (256, 512)), ("pfc", (136, 200)), ("pfc", (64, 64)),
                                        ("pfc", (1000, 1002)), ("cdft", (64, 128))])
def test_tensor_copy_staging_equals_cp_async_staging(kind, shape, precision, monkeypatch):
    """Variants 27..29 stage each tile with one tensor copy per array (zeros
    outside the grid, then the wrapped values by plain loads) and run the same
    updates as 24, 0 and 26, so the results agree bit for bit: on a grid of
    interior and boundary tiles, a ragged one, one where every tile crosses
    the periodic boundary, and one whose rows are not a whole number of 16
    bytes (staged by cp.async there); 2 and 3 sweeps."""
    monkeypatch.setenv("FM_RB_VARIANT", "0")  # no autotuning at create
    rho, vel, prm = _case(kind, shape, 11)
    f, _ = _oracle(rho, vel, prm, 0.0, 0)
    for sweeps in (2, 3):
        for vt, vc in ((27, 24), (28, 0), (29, 26)):
            try:
                ref = _gpu(rho, vel, prm, f, precision, 0.0, sweeps, vc)
                tma = _gpu(rho, vel, prm, f, precision, 0.0, sweeps, vt)
            except fm.FMError as err:
                assert err.code == fm.FM_EINVAL and precision == fm.FM_FP64
                continue
            for q, (a, b) in enumerate(zip(tma, ref)):
                assert np.array_equal(a, b), (sweeps, vt, q, float(np.max(np.abs(a - b))))


def _case3(kind, shape, seed):
    rng = np.random.default_rng(seed)
    if kind == "cdft":
        rho = 0.3 + 0.05 * rng.uniform(0, 1, shape)
        prm = dict(kind="cdft", dim=3, h=17.0 / shape[2], dt=0.02, nu=2.362, delta=1e-10)
    else:
        rho = 0.8 + 0.05 * rng.uniform(-1, 1, shape)
        prm = dict(kind="pfc", dim=3, h=0.9, dt=0.02, alpha=0.6)
    vel = [0.05 * rng.standard_normal(shape) for _ in range(3)]
    return rho, vel, prm


@pytest.mark.parametrize("precision", [fm.FM_FP64, fm.FM_MIXED])
@pytest.mark.parametrize("kind,shape", [("pfc", (24, 48, 96)), ("pfc", (128, 64, 64)), ("pfc", (4, 16, 32)),
                                        ("pfc", (2, 16, 64)), ("cdft", (16, 32, 32))])
def test_3d_z_marching_sweeps_equal_colour_launches(kind, shape, precision, monkeypatch):
    """The z-marching 3-D sweeps (variants 3 and 4: tiles of 32 x 8 and
    32 x 16 points, planes staged in shared memory) run the point update of
    the red and the black launch on the same values, so they agree with the
    two-colour sweeps to the rounding of the compiled point update (the
    tolerances of the 2-D variants; measured: float64 bit for bit, float32
    within a few ulps): several tiles in x and y, the x rows of
    the last tile wrapping around, blocks whose share of the planes is cut at
    arbitrary planes and crosses tiles (64 x 64 x 128: about seven planes per
    block), four and two planes (the staged planes wrap around z), and CDFT
    (the coefficient density staged as well); 1 and 3 sweeps.  Where a tile
    does not fit (32 x 16 float64) the variant falls back to the colour
    launches."""
    monkeypatch.setenv("FM_RB_VARIANT", "0")  # no autotuning at create
    rho, vel, prm = _case3(kind, shape, 13)
    f, _ = _oracle(rho, vel, prm, 0.0, 0)
    tol = 1e-12 if precision == fm.FM_FP64 else 2e-5
    for sweeps in (1, 3):
        ref = _gpu(rho, vel, prm, f, precision, 0.0, sweeps, fm.FM_SWEEP_TWO_COLOUR)
        assert max(float(np.max(np.abs(x))) for x in ref) > 0
        for v in (3, 4):
            _close(_gpu(rho, vel, prm, f, precision, 0.0, sweeps, v), ref, tol)


def test_smooth_row_rejects_bad_arguments():
    rho, vel, prm = _case("cdft", (32, 32), 7)
    sol = gpu_solver(rho, prm)
    sol.set_fields(rho, vel)
    e = [np.zeros_like(rho) for _ in range(3)]
    with pytest.raises(fm.FMError):  # before fm_prepare
        fm.fm_smooth(sol.handle, e, e, 1)
    fm.fm_prepare(sol.handle, prm["dt"])
    for variant in (-3, fm.FM_SWEEP_VARIANTS):
        with pytest.raises(fm.FMError):
            fm.fm_smooth(sol.handle, e, e, 1, variant)
    with pytest.raises(fm.FMError):
        fm.fm_smooth(sol.handle, e, e, -1)
    fm.fm_smooth(sol.handle, e, e, 0)
    sol.close()


@pytest.mark.parametrize("precision", [fm.FM_FP64, fm.FM_MIXED])
def test_cdft_sweeps_match_oracle_where_the_projection_is_active(precision):
    """Near vacuum the positive projection of Sec. 6 decides the update: a
    Gaussian blob on a floor of 1e-10 = delta puts every density outside the
    blob at the order of delta, where sqrt(rho^2 + delta^2) moves rho by tens
    of percent.  Three sweeps (w = 0.5) against the oracle's, element by
    element as above, and relatively at the near-vacuum points themselves,
    where a smoother without the projection would be 30-40% off."""
    n = 64
    L = 34.0
    h = L / n
    x = np.arange(n) * h
    X, Y = np.meshgrid(x, x, indexing="xy")
    rho = 1e-10 + 0.5 * np.exp(-((X - L / 2) ** 2 + (Y - L / 2) ** 2) / (2 * (L / 16) ** 2))
    rng = np.random.default_rng(8)
    vel = [0.05 * np.sin(2 * np.pi * X / L) * np.cos(2 * np.pi * Y / L) + 0.01 * rng.standard_normal((n, n)),
           0.05 * np.cos(2 * np.pi * X / L) * np.sin(2 * np.pi * Y / L)]
    prm = dict(kind="cdft", dim=2, h=h, dt=0.02, nu=2.362, delta=1e-10)
    f, de = _oracle(rho, vel, prm, 0.5, 3)
    e = _gpu(rho, vel, prm, f, precision, 0.5, 3, fm.FM_SWEEP_AUTO)
    _close(e, de, TOL[precision])
    vac = rho < 1e-9
    assert vac.sum() > n * n // 4
    new_o = rho + de[0]
    new_g = rho + e[0]
    assert np.all(new_o[vac] > 1.3e-10)  # the projection moved every near-vacuum density
    err = np.max(np.abs(new_g[vac] - new_o[vac]) / new_o[vac])
    assert err <= (1e-10 if precision == fm.FM_FP64 else 1e-4), err
