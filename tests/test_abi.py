"""The C-ABI library builds, loads and exports every symbol include/fm.h
declares; host-side argument checks reject bad input before any CUDA call.
No compute runs here (no GPU needed)."""
import ctypes as C
import os
import re

import pytest

from paper_1503_07416_gb300 import build, fm

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "fm.h")


@pytest.fixture(scope="module")
def lib():
    build.build_library()
    return fm.lib()


def declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(fm_[a-z0-9_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    names = declared()
    assert "fm_create" in names and "fm_step" in names and "fm_energy" in names and "fm_mass" in names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    # and the binding wraps each of them under the same name
    assert all(hasattr(fm, n) for n in names)


def test_default_params_and_strerror(lib):
    p = fm.fm_default_params()
    assert p.gamma == 2.0 and p.nu1 == 2 and p.nu2 == 2 and p.sigma == 1.0
    assert p.precision == fm.FM_FP64 and p.tol == 1e-10
    assert p.coarse_precision == fm.FM_FP64  # the coarsest-grid solve of the mixed path in float64
    codes = (fm.FM_OK, fm.FM_EINVAL, fm.FM_ENOMEM, fm.FM_ECUDA, fm.FM_ENOCONV, fm.FM_ENONPOS, fm.FM_ENAN,
             fm.FM_ETIMEOUT)
    msgs = [fm.strerror(code) for code in codes]
    assert all(isinstance(m, str) and m and m != "unknown error" for m in msgs)
    assert len(set(msgs)) == len(codes)


def _create(dim=2, n=(8, 8, 1), h=0.5, kind=fm.FM_PFC, nu=1.0, **kw):
    g = fm.fm_grid()
    g.dim = dim
    for d in range(3):
        g.n[d] = n[d]
    g.h = h
    f = fm.fm_functional()
    f.kind = kind
    f.alpha = 0.6
    f.nu = nu
    p = fm.fm_default_params()
    for k, v in kw.items():
        setattr(p, k, v)
    h_ = C.c_void_p()
    return fm.lib().fm_create(C.byref(g), C.byref(p), C.byref(f), C.byref(h_))


@pytest.mark.parametrize("bad", [
    dict(dim=4), dict(n=(7, 8, 1)), dict(n=(0, 8, 1)), dict(h=0.0), dict(kind=9),
    dict(kind=fm.FM_CDFT, n=(12, 8, 1)), dict(kind=fm.FM_CDFT, nu=0.0), dict(tol=0.0),
    dict(w_damp=1.0), dict(nu1=0, nu2=0), dict(ncoarse=0), dict(precision=7), dict(coarsest=1),
    dict(dim=3, n=(8, 8, 5)), dict(model=7), dict(walls=3), dict(init=5),
    dict(walls=1, kind=fm.FM_CDFT, n=(8, 8, 1)), dict(walls=1, dim=3, n=(8, 8, 8)),
    dict(init=1, model=1), dict(coarse_precision=3), dict(coarse_precision=-1),
])
def test_create_rejects_invalid_arguments(lib, bad):
    assert _create(**bad) == fm.FM_EINVAL


def test_null_handles_are_rejected(lib):
    L = fm.lib()
    assert L.fm_step(None, C.c_double(0.1), None) == fm.FM_EINVAL
    assert L.fm_mass(None, None) == fm.FM_EINVAL
    assert L.fm_set_stream(None, None) == fm.FM_EINVAL
    L.fm_destroy(None)


def test_mass_noalloc_rejects_oversized_grids_before_any_cuda_call(lib):
    """Sizes whose product overflows 64 bits, or exceeds the static scratch,
    are rejected by the host-side checks (the pointers are never touched)."""
    L = fm.lib()
    fake = C.c_void_p(0x1000)
    for dims, n in ((3, (2 ** 31 - 1, 2 ** 31 - 1, 2 ** 31 - 1)), (2, (4096, 1025, 1)),
                    (3, (1 << 20, 1 << 20, 4)), (2, (0, 8, 1))):
        arr = (C.c_int * 3)(*n)
        assert L.fm_mass_noalloc(fake, dims, arr, C.c_double(1.0), fake, None) == fm.FM_EINVAL


def test_mass_noalloc_wrapper_checks_its_arguments(lib):
    """The binding raises ValueError for host arrays, CPU tensors, float32
    tensors and non-contiguous views before calling the library."""
    import numpy as np
    torch = pytest.importorskip("torch")
    out_cpu = torch.zeros(1, dtype=torch.float64)
    with pytest.raises(ValueError):
        fm.fm_mass_noalloc(np.zeros((8, 8)), 1.0, out_cpu)
    with pytest.raises(ValueError):
        fm.fm_mass_noalloc(torch.zeros((8, 8), dtype=torch.float64), 1.0, out_cpu)
    with pytest.raises(ValueError):
        fm.fm_mass_noalloc(torch.zeros((8, 8), dtype=torch.float32), 1.0, out_cpu)


def test_grid_barrier_selftest_rejects_limits_out_of_range(lib):
    """Checked before any device work (no GPU needed)."""
    for limit in (0, -5, 1000001):
        assert fm.fm_grid_barrier_selftest(True, limit) == fm.FM_EINVAL


def test_wait_selftest_rejects_limits_out_of_range(lib):
    """Checked before any device work (no GPU needed)."""
    for limit in (0, -5, 1000001):
        assert fm.fm_wait_selftest(True, limit) == fm.FM_EINVAL
