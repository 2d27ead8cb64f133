"""Batched ensembles (fm_create_batch / fm_step_batch) against the oracle and
against single-instance steps, with uneven grid sizes and per-instance time
steps.  Tolerances as in test_gpu_parity (float64 1e-10, mixed 1e-8 relative
per field against the oracle)."""
import functools
import math

import numpy as np
import pytest

from oracle import scheme as S
from paper_1503_07416_gb300 import fm, inputs
from tests.helpers import assert_parity, gpu_solver, oracle_setup, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1503_07416_gb300 import build
    build.build_library()
    fm.lib()


def _ensemble(kind, sizes, seed):
    rng = np.random.default_rng(seed)
    states = []
    for k, n in enumerate(sizes):
        shape = tuple(reversed(n)) if isinstance(n, tuple) else (n, n)
        if kind == "pfc":
            rho = 0.8 + 0.05 * rng.uniform(-1, 1, shape)
        else:
            rho = 0.1 * math.pi * (1 + 0.1 * rng.uniform(0, 1, shape))
        vel = [0.03 * rng.standard_normal(shape) for _ in range(2)]
        dt = float(math.exp(rng.uniform(math.log(1e-3), math.log(5e-2))))
        states.append((rho, vel, dt))
    return states


@pytest.mark.parametrize("precision", [fm.FM_FP64, fm.FM_MIXED])
def test_batch_pfc_uneven_sizes(precision):
    """Six PFC instances of sizes 16^2 .. 128^2 and a ragged 48x40, each with
    its own dt, two steps; every instance matches the oracle and the
    single-instance solver."""
    sizes = [16, 32, (48, 40), 64, 128, 32]
    ens = _ensemble("pfc", sizes, 5)
    h, tol = 0.9, 1e-12
    prm = dict(kind="pfc", dim=2, h=h, alpha=0.6, tol=tol)
    b = fm.Batch("pfc", sizes, h, alpha=0.6, precision=precision, tol=tol, w_damp=0.0, max_cycles=80)
    for i, (rho, vel, dt) in enumerate(ens):
        b.set_fields(i, rho, vel)
    bound = 1e-10 if precision == fm.FM_FP64 else 1e-8
    cur = [(r, v) for r, v, _ in ens]
    for step in range(2):
        info = b.step([dt for _, _, dt in ens])
        for i, (rho, vel, dt) in enumerate(ens):
            assert info[i].res <= tol
            rg, vg = b.get_fields(i)
            P, opts, J = oracle_setup(cur[i][0], dict(prm, dt=dt), w_damp=0.0, tol=tol)
            ro, vo, _ = S.step(cur[i][0], cur[i][1], P, opts, J=J)
            assert_parity(rg, vg, ro, vo, bound, (i, step))
            # single-instance path from the same state
            sol = gpu_solver(cur[i][0], dict(prm, dt=dt), precision=precision, w_damp=0.0, tol=tol)
            sol.set_fields(cur[i][0], cur[i][1])
            sinfo = sol.step(dt)
            rs, vs = sol.get_fields()
            sol.close()
            assert sinfo.cycles == info[i].cycles
            assert rel(rg, rs) <= 1e-12 and all(rel(a, c) <= 1e-12 for a, c in zip(vg, vs))
            cur[i] = (rg, vg)
    b.close()


def test_batch_cdft():
    """Three CDFT instances (power-of-two sizes) with their own dt."""
    sizes = [16, 32, 64]
    ens = _ensemble("cdft", sizes, 7)
    tol = 1e-12
    out = []
    b = fm.Batch("cdft", sizes, 34.0 / 128, nu=2.362, precision=fm.FM_MIXED, tol=tol, w_damp=0.5,
                 delta=1e-10, max_cycles=80)
    for i, (rho, vel, dt) in enumerate(ens):
        b.set_fields(i, rho, vel)
    info = b.step([dt for _, _, dt in ens])
    for i, (rho, vel, dt) in enumerate(ens):
        prm = dict(kind="cdft", dim=2, h=34.0 / 128, nu=2.362, delta=1e-10, dt=dt)
        P, opts, J = oracle_setup(rho, prm, w_damp=0.5, tol=tol)
        ro, vo, _ = S.step(rho, vel, P, opts, J=J)
        rg, vg = b.get_fields(i)
        assert_parity(rg, vg, ro, vo, 1e-8, i)
    b.close()


def test_batch_failure_is_isolated():
    """A NaN in one instance makes that instance report FM_ENAN and keep its
    state; the others advance normally."""
    sizes = [32, 32, 64]
    ens = _ensemble("pfc", sizes, 9)
    b = fm.Batch("pfc", sizes, 0.9, alpha=0.6, precision=fm.FM_MIXED, tol=1e-10, w_damp=0.0)
    bad = ens[1][0].copy()
    bad[3, 4] = math.nan
    for i, (rho, vel, dt) in enumerate(ens):
        b.set_fields(i, bad if i == 1 else rho, vel)
    code, info = fm.fm_step_batch(b.handle, [dt for _, _, dt in ens])
    assert code == fm.FM_ENAN
    r1, v1 = b.get_fields(1)
    assert np.isnan(r1[3, 4]) and np.array_equal(v1[0], ens[1][1][0])
    for i in (0, 2):
        assert info[i].res <= 1e-10
        r, _ = b.get_fields(i)
        assert not np.array_equal(r, ens[i][0])
    b.close()


@pytest.mark.parametrize("variant", [21, 24])
@pytest.mark.parametrize("nu", [(2, 2), (1, 3), (3, 2)])
@pytest.mark.parametrize("precision", [fm.FM_FP64, fm.FM_MIXED])
def test_batch_two_sweep_smoother(precision, nu, variant, monkeypatch):
    """The batch with a two-sweep variant (marching 21, tile 24) on every level: the
    correction of a level may sit in its second buffer between the pre- and
    the post-smoothing (the fused residual + restriction and the prolongation
    take it from there) and an odd sweep count runs the one-sweep variant of
    the same blocks.  Against the oracle with the same cycle and the
    single-instance solver with the same variant."""
    monkeypatch.setenv("FM_RB_VARIANT", str(variant))
    sizes = [32, (256, 192), 128]
    ens = _ensemble("pfc", sizes, 12)
    h, tol = 0.9, 1e-12
    prm = dict(kind="pfc", dim=2, h=h, alpha=0.6, tol=tol)
    b = fm.Batch("pfc", sizes, h, alpha=0.6, precision=precision, tol=tol, w_damp=0.0, max_cycles=80,
                 nu1=nu[0], nu2=nu[1])
    for i, (rho, vel, dt) in enumerate(ens):
        b.set_fields(i, rho, vel)
    info = b.step([dt for _, _, dt in ens])
    bound = 1e-10 if precision == fm.FM_FP64 else 1e-8
    for i, (rho, vel, dt) in enumerate(ens):
        assert info[i].res <= tol
        rg, vg = b.get_fields(i)
        P, opts, J = oracle_setup(rho, dict(prm, dt=dt), w_damp=0.0, tol=tol)
        opts.nu1, opts.nu2 = nu
        ro, vo, _ = S.step(rho, vel, P, opts, J=J)
        assert_parity(rg, vg, ro, vo, bound, i)
        sol = gpu_solver(rho, dict(prm, dt=dt), precision=precision, w_damp=0.0, tol=tol, nu1=nu[0], nu2=nu[1])
        sol.set_fields(rho, vel)
        sol.step(dt)
        rs, vs = sol.get_fields()
        sol.close()
        assert rel(rg, rs) <= 1e-12 and all(rel(a, c) <= 1e-12 for a, c in zip(vg, vs))
    b.close()


@pytest.mark.parametrize("precision", [fm.FM_FP64, fm.FM_MIXED])
def test_batch_odd_sweep_counts(precision):
    """V(1,3): every smoothing stage has an odd number of fused sweeps, so the
    batch copies the correction back after the last one; two instances (one
    of them several tile waves large) against the oracle with the same cycle
    and against the single-instance solver."""
    sizes = [32, (256, 192)]
    ens = _ensemble("pfc", sizes, 11)
    h, tol = 0.9, 1e-12
    prm = dict(kind="pfc", dim=2, h=h, alpha=0.6, tol=tol)
    b = fm.Batch("pfc", sizes, h, alpha=0.6, precision=precision, tol=tol, w_damp=0.0, max_cycles=80,
                 nu1=1, nu2=3)
    for i, (rho, vel, dt) in enumerate(ens):
        b.set_fields(i, rho, vel)
    info = b.step([dt for _, _, dt in ens])
    bound = 1e-10 if precision == fm.FM_FP64 else 1e-8
    for i, (rho, vel, dt) in enumerate(ens):
        assert info[i].res <= tol
        rg, vg = b.get_fields(i)
        P, opts, J = oracle_setup(rho, dict(prm, dt=dt), w_damp=0.0, tol=tol)
        opts.nu1, opts.nu2 = 1, 3
        ro, vo, _ = S.step(rho, vel, P, opts, J=J)
        assert_parity(rg, vg, ro, vo, bound, i)
        sol = gpu_solver(rho, dict(prm, dt=dt), precision=precision, w_damp=0.0, tol=tol, nu1=1, nu2=3)
        sol.set_fields(rho, vel)
        sol.step(dt)
        rs, vs = sol.get_fields()
        sol.close()
        assert rel(rg, rs) <= 1e-12 and all(rel(a, c) <= 1e-12 for a, c in zip(vg, vs))
    b.close()


@pytest.mark.parametrize("precision", [fm.FM_FP64, fm.FM_MIXED])
def test_batch_with_the_benchmark_hierarchy(precision):
    """The hierarchy the batch benchmark uses (coarsest 64, two coarse sweeps):
    the 64 x 64 and 96 x 64 coarsest levels are too large for the
    shared-memory coarse kernel, so the batch takes the global-memory one."""
    sizes = [128, (192, 128)]
    ens = _ensemble("pfc", sizes, 13)
    h, tol = 0.9, 1e-12
    prm = dict(kind="pfc", dim=2, h=h, alpha=0.6, tol=tol)
    b = fm.Batch("pfc", sizes, h, alpha=0.6, precision=precision, tol=tol, w_damp=0.0, max_cycles=80,
                 **inputs.BENCH_MG_2D)
    for i, (rho, vel, dt) in enumerate(ens):
        b.set_fields(i, rho, vel)
    info = b.step([dt for _, _, dt in ens])
    bound = 1e-10 if precision == fm.FM_FP64 else 1e-8
    for i, (rho, vel, dt) in enumerate(ens):
        assert info[i].res <= tol
        rg, vg = b.get_fields(i)
        P, opts, J = oracle_setup(rho, dict(prm, dt=dt), w_damp=0.0, tol=tol)
        ro, vo, _ = S.step(rho, vel, P, opts, J=J)
        assert_parity(rg, vg, ro, vo, bound, i)
    b.close()


def test_batch_smoother_timing_entry_points():
    """fm_batch_time_smoother times the autotuned variant and
    fm_batch_time_sweep_variant any fixed one (positive times, the finest
    points of the multi-kernel instances); unknown variants are rejected, and
    a later step still converges (the timed sweeps only touch scratch)."""
    sizes = [128, 256]
    ens = _ensemble("pfc", sizes, 13)
    b = fm.Batch("pfc", sizes, 0.9, alpha=0.6, precision=fm.FM_MIXED, tol=1e-10, w_damp=0.0, max_cycles=80)
    for i, (rho, vel, dt) in enumerate(ens):
        b.set_fields(i, rho, vel)
    ms, pts = fm.fm_batch_time_smoother(b.handle, 3)
    assert ms > 0 and pts == 128 * 128 + 256 * 256
    for v in (0, 16, 22, 24):
        ms_v, pts_v = fm.fm_batch_time_sweep_variant(b.handle, v, 3)
        assert ms_v > 0 and pts_v == pts
    for v in (-1, fm.FM_SWEEP_VARIANTS):
        with pytest.raises(fm.FMError):
            fm.fm_batch_time_sweep_variant(b.handle, v, 3)
    info = b.step([dt for _, _, dt in ens])
    assert all(x.res <= 1e-10 for x in info)
    b.close()


BIG_SIZES = [1024, 128, 512, 256, 64, 256, 128, 512, 128, 256]


@functools.lru_cache(maxsize=1)
def _big_ensemble():
    """Ten instances with the benchmark ensemble's physics (eps = 0.4,
    supercooled liquid with nuclei, h = pi/(2 sqrt 3)), one of them 1024^2,
    seeded velocities and per-instance dt log-uniform in [1e-3, 1e-1], and
    one oracle step of each (shared by both precisions)."""
    rng = np.random.default_rng(31)
    out = []
    for k, n in enumerate(BIG_SIZES):
        rho, _, prm = inputs.pfc_supercooled(n, seed=500 + k)
        vel = [0.02 * rng.standard_normal(rho.shape) for _ in range(2)]
        dt = float(math.exp(rng.uniform(math.log(1e-3), math.log(1e-1))))
        prm = dict(prm, dt=dt)
        P, opts, J = oracle_setup(rho, prm, w_damp=0.0, tol=1e-11)
        ro, vo, _ = S.step(rho, vel, P, opts, J=J)
        out.append((rho, vel, prm, ro, vo))
    return out


@pytest.mark.parametrize("precision", [fm.FM_FP64, fm.FM_MIXED])
def test_batch_ten_instances_with_a_1024_grid(precision):
    """A batch of more than eight instances holding a 1024^2 grid, in the
    benchmark's configuration (undamped, the benchmark hierarchy): every
    instance against its own oracle step, element by element."""
    ens = _big_ensemble()
    p0 = ens[0][2]
    b = fm.Batch("pfc", BIG_SIZES, p0["h"], alpha=p0["alpha"], precision=precision, tol=1e-11, w_damp=0.0,
                 max_cycles=80, **inputs.BENCH_MG_2D)
    for i, (rho, vel, _, _, _) in enumerate(ens):
        b.set_fields(i, rho, vel)
    info = b.step([e[2]["dt"] for e in ens])
    bound = 1e-10 if precision == fm.FM_FP64 else 1e-8
    for i, (_, _, _, ro, vo) in enumerate(ens):
        assert info[i].res <= 1e-11, (i, info[i].res)
        rg, vg = b.get_fields(i)
        assert_parity(rg, vg, ro, vo, bound, (i, BIG_SIZES[i]))
    b.close()


def test_batch48_full_ensemble_sampled():
    """The whole 48-instance benchmark ensemble (15.4 M points, mixed, the
    benchmark hierarchy, tol 1e-10) stepped once as the benchmark steps it;
    the oracle recomputes a sample -- the first instance of each grid size
    and two seeded picks -- and each sampled instance must match it element
    by element; every instance must have converged and conserved mass."""
    ens = inputs.batch48()
    sizes = [prm["n"] for _, _, prm in ens]
    p0 = ens[0][2]
    b = fm.Batch("pfc", sizes, p0["h"], alpha=p0["alpha"], precision=fm.FM_MIXED, tol=p0["tol"], w_damp=0.0,
                 gamma=p0["gamma"], delta=0.0, **inputs.BENCH_MG_2D)
    for i, (rho, vel, _) in enumerate(ens):
        b.set_fields(i, rho, vel)
    info = b.step([prm["dt"] for _, _, prm in ens])
    sample = sorted({sizes.index(n) for n in set(sizes)} |
                    set(int(x) for x in np.random.default_rng(48).choice(len(ens), 2, replace=False)))
    for i, (rho, vel, prm) in enumerate(ens):
        assert info[i].res <= prm["tol"], (i, info[i].res)
        rg, vg = b.get_fields(i)
        assert abs(rg.sum() - rho.sum()) <= 1e-12 * rho.sum(), i
        if i in sample:
            P, opts, J = oracle_setup(rho, prm, w_damp=0.0, tol=prm["tol"])
            ro, vo, _ = S.step(rho, vel, P, opts, J=J)
            assert_parity(rg, vg, ro, vo, 1e-8, (i, sizes[i]))
    b.close()


def test_batch_nonpositive_instance_is_isolated():
    """A CDFT instance whose density is <= 0 somewhere reports FM_ENONPOS and
    keeps its state; the other instances advance."""
    sizes = [32, 32, 64]
    ens = _ensemble("cdft", sizes, 19)
    b = fm.Batch("cdft", sizes, 34.0 / 128, nu=2.362, precision=fm.FM_MIXED, tol=1e-10, w_damp=0.5,
                 delta=1e-10, max_cycles=80)
    bad = ens[1][0].copy()
    bad[4, 9] = -0.05
    for i, (rho, vel, dt) in enumerate(ens):
        b.set_fields(i, bad if i == 1 else rho, vel)
    code, info = fm.fm_step_batch(b.handle, [dt for _, _, dt in ens])
    assert code == fm.FM_ENONPOS
    r1, v1 = b.get_fields(1)
    assert np.array_equal(r1, bad) and np.array_equal(v1[0], ens[1][1][0])
    for i in (0, 2):
        assert info[i].res <= 1e-10
        r, _ = b.get_fields(i)
        assert not np.array_equal(r, ens[i][0])
    # the flag is cleared at the next step
    b.set_fields(1, ens[1][0], ens[1][1])
    code, info = fm.fm_step_batch(b.handle, [dt for _, _, dt in ens])
    assert code == fm.FM_OK
    b.close()
