"""ctypes binding of libfm (include/fm.h): argument marshalling only.

Every function here has the name of the C entry point it calls.  Arrays may be
numpy float64 arrays (host memory) or torch float64 CUDA tensors (device
memory); every step of the computation runs in the CUDA library.  Loading
fails loudly when libfm.so is missing: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIBPATH = os.path.join(_PKG, "libfm.so")

FM_OK = 0
FM_EINVAL = -1
FM_ENOMEM = -2
FM_ECUDA = -3
FM_ENOCONV = -4
FM_ENONPOS = -5
FM_ENAN = -6
FM_ETIMEOUT = -7
FM_PFC = 1
FM_CDFT = 2
FM_FP64 = 0
FM_MIXED = 1
FM_HOST = 0
FM_DEVICE = 1
FM_HYDRO = 0
FM_GRADFLOW = 1
FM_WALLS_NONE = 0
FM_WALLS_Y = 1
FM_INIT_PREVIOUS = 0
FM_INIT_EXTRAPOLATE = 1
FM_AUX_OMEGA = 1
FM_AUX_SOURCE = 2
FM_AUX_CONV = 3
FM_AUX_ITERATE = 4


class fm_grid(C.Structure):
    _fields_ = [("dim", C.c_int), ("n", C.c_int * 3), ("h", C.c_double)]


class fm_functional(C.Structure):
    _fields_ = [("kind", C.c_int), ("alpha", C.c_double), ("nu", C.c_double)]


class fm_params(C.Structure):
    _fields_ = [("gamma", C.c_double), ("w_damp", C.c_double), ("delta", C.c_double),
                ("tol", C.c_double), ("sigma", C.c_double), ("nu1", C.c_int), ("nu2", C.c_int),
                ("max_cycles", C.c_int), ("coarsest", C.c_int), ("ncoarse", C.c_int),
                ("precision", C.c_int), ("model", C.c_int), ("walls", C.c_int), ("u_wall", C.c_double * 2),
                ("init", C.c_int), ("coarse_precision", C.c_int)]


class fm_step_info(C.Structure):
    _fields_ = [("cycles", C.c_int), ("res0", C.c_double), ("res", C.c_double)]


class FMError(RuntimeError):
    def __init__(self, code, what):
        super().__init__(f"{what}: {strerror(code)} ({code})")
        self.code = code


_lib = None

_SIGS = {
    "fm_default_params": (None, [C.POINTER(fm_params)]),
    "fm_create": (C.c_int, [C.POINTER(fm_grid), C.POINTER(fm_params), C.POINTER(fm_functional),
                            C.POINTER(C.c_void_p)]),
    "fm_destroy": (None, [C.c_void_p]),
    "fm_set_stream": (C.c_int, [C.c_void_p, C.c_void_p]),
    "fm_set_fields": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(C.c_void_p), C.c_int]),
    "fm_get_fields": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(C.c_void_p), C.c_int]),
    "fm_step": (C.c_int, [C.c_void_p, C.c_double, C.POINTER(fm_step_info)]),
    "fm_step_host": (C.c_int, [C.c_void_p, C.c_double, C.c_void_p, C.POINTER(C.c_void_p), C.c_void_p,
                               C.POINTER(C.c_void_p), C.POINTER(fm_step_info)]),
    "fm_energy": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_double),
                            C.POINTER(C.c_double)]),
    "fm_mass": (C.c_int, [C.c_void_p, C.POINTER(C.c_double)]),
    "fm_energy_terms": (C.c_int, [C.c_void_p, C.POINTER(C.c_double)]),
    "fm_strerror": (C.c_char_p, [C.c_int]),
    "fm_prepare": (C.c_int, [C.c_void_p, C.c_double]),
    "fm_get_aux": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_int]),
    "fm_residual": (C.c_int, [C.c_void_p, C.POINTER(C.c_void_p), C.POINTER(C.c_void_p),
                              C.POINTER(C.c_double), C.c_int]),
    "fm_convolve": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]),
    "fm_restrict": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]),
    "fm_prolong_add": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]),
    "fm_levels": (C.c_int, [C.c_void_p]),
    "fm_narrow": (C.c_int, [C.c_void_p, C.c_void_p, C.c_longlong, C.c_void_p]),
    "fm_widen": (C.c_int, [C.c_void_p, C.c_void_p, C.c_longlong, C.c_void_p]),
    "fm_wait_selftest": (C.c_int, [C.c_int, C.c_int, C.c_void_p]),
    "fm_grid_barrier_selftest": (C.c_int, [C.c_int, C.c_int, C.c_void_p]),
    "fm_smooth": (C.c_int, [C.c_void_p, C.POINTER(C.c_void_p), C.POINTER(C.c_void_p), C.c_int, C.c_int, C.c_int]),
    "fm_create_batch": (C.c_int, [C.c_int, C.POINTER(fm_grid), C.POINTER(fm_params), C.POINTER(fm_functional),
                                  C.POINTER(C.c_void_p)]),
    "fm_destroy_batch": (None, [C.c_void_p]),
    "fm_batch_set_stream": (C.c_int, [C.c_void_p, C.c_void_p]),
    "fm_batch_instance": (C.c_void_p, [C.c_void_p, C.c_int]),
    "fm_step_batch": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.POINTER(fm_step_info)]),
    "fm_batch_launches": (C.c_longlong, [C.c_void_p]),
    "fm_batch_tuning": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_float)]),
    "fm_batch_time_smoother": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_longlong)]),
    "fm_batch_time_sweep_variant": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.POINTER(C.c_double),
                                              C.POINTER(C.c_longlong)]),
    "fm_mass_noalloc": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_int), C.c_double, C.c_void_p,
                                  C.c_void_p]),
    "fm_profile": (C.c_int, [C.c_void_p, C.c_int]),
    "fm_tuning": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_float)]),
    "fm_profile_read": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_longlong),
                                  C.POINTER(C.c_longlong)]),
}


def lib():
    """Load libfm.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIBPATH):
            raise RuntimeError(f"libfm.so not found at {LIBPATH}: build it with "
                               "python -m paper_1503_07416_gb300.build")
        L = C.CDLL(LIBPATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def fm_strerror(code):
    return lib().fm_strerror(code).decode()


strerror = fm_strerror


def _check(code, what):
    if code != FM_OK:
        raise FMError(code, what)


def _ptr(a):
    """(address, where) of a float64 numpy array or torch tensor."""
    if isinstance(a, np.ndarray):
        if a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"]:
            raise ValueError("host arrays must be C-contiguous float64")
        return a.ctypes.data, FM_HOST
    import torch  # noqa: F401  (device arrays are torch tensors)
    if a.dtype != torch.float64 or not a.is_contiguous():
        raise ValueError("device tensors must be contiguous float64")
    return a.data_ptr(), (FM_DEVICE if a.is_cuda else FM_HOST)


def _where(arrs):
    ws = {_ptr(a)[1] for a in arrs if a is not None}
    if len(ws) != 1:
        raise ValueError("mix of host and device arrays")
    return ws.pop()


def _vec(arrs):
    return (C.c_void_p * len(arrs))(*[(_ptr(a)[0] if a is not None else None) for a in arrs])


def fm_default_params():
    p = fm_params()
    lib().fm_default_params(C.byref(p))
    return p


def fm_create(grid: fm_grid, prm: fm_params, fn: fm_functional):
    h = C.c_void_p()
    _check(lib().fm_create(C.byref(grid), C.byref(prm), C.byref(fn), C.byref(h)), "fm_create")
    return h


def fm_destroy(st):
    lib().fm_destroy(st)


def fm_set_stream(st, stream_handle: int):
    _check(lib().fm_set_stream(st, C.c_void_p(stream_handle)), "fm_set_stream")


def fm_set_fields(st, rho, vel):
    """vel may be None (gradient-flow states have no velocity)."""
    vel = list(vel) if vel is not None else []
    w = _where([rho, *vel])
    _check(lib().fm_set_fields(st, C.c_void_p(_ptr(rho)[0]), _vec(vel) if vel else None, w), "fm_set_fields")


def fm_get_fields(st, rho, vel):
    w = _where([rho, *vel])
    _check(lib().fm_get_fields(st, C.c_void_p(_ptr(rho)[0]), _vec(vel), w), "fm_get_fields")


def fm_step(st, dt):
    info = fm_step_info()
    _check(lib().fm_step(st, C.c_double(dt), C.byref(info)), "fm_step")
    return info


def fm_step_host(st, dt, rho_in, vel_in, rho_out, vel_out):
    """fm_step_host: one step of host-resident fields (numpy or CPU tensors,
    float64, C-contiguous); returns (code, info) without raising.  vel_in and
    vel_out may be None for gradient-flow states."""
    info = fm_step_info()
    code = lib().fm_step_host(st, C.c_double(dt), C.c_void_p(_ptr(rho_in)[0]),
                              _vec(vel_in) if vel_in else None, C.c_void_p(_ptr(rho_out)[0]),
                              _vec(vel_out) if vel_out else None, C.byref(info))
    return code, info


class HostStepper:
    """Repeated fm_step_host calls on the same host buffers (see
    Solver.host_stepper).  The buffers must stay alive and unmoved; the
    returned fm_step_info is overwritten by the next call."""

    def __init__(self, sol, rho_in, vel_in, rho_out, vel_out):
        arrs = [rho_in, *vel_in, rho_out, *vel_out]
        for a in arrs:
            if _ptr(a)[1] != FM_HOST:
                raise ValueError("fm_step_host takes host arrays")
        self._keep = arrs
        self._handle = sol.handle
        self._args = (C.c_void_p(_ptr(rho_in)[0]), _vec(vel_in), C.c_void_p(_ptr(rho_out)[0]), _vec(vel_out))
        self._info = fm_step_info()
        self._fn = lib().fm_step_host

    def __call__(self, dt):
        _check(self._fn(self._handle, C.c_double(dt), *self._args, C.byref(self._info)), "fm_step_host")
        return self._info


def fm_step_raw(st, dt):
    """fm_step returning (code, info) without raising."""
    info = fm_step_info()
    code = lib().fm_step(st, C.c_double(dt), C.byref(info))
    return code, info


def fm_energy(st):
    E, F, K = C.c_double(), C.c_double(), C.c_double()
    _check(lib().fm_energy(st, C.byref(E), C.byref(F), C.byref(K)), "fm_energy")
    return E.value, F.value, K.value


def fm_energy_terms(st):
    """[KE, then the PFC terms (quartic, quadratic, (Lap rho)^2/2, rho Lap rho)
    or CDFT (F_id, F_ex, 0, 0)]."""
    t = (C.c_double * 5)()
    _check(lib().fm_energy_terms(st, t), "fm_energy_terms")
    return list(t)


def fm_mass(st):
    M = C.c_double()
    _check(lib().fm_mass(st, C.byref(M)), "fm_mass")
    return M.value


def fm_prepare(st, dt):
    _check(lib().fm_prepare(st, C.c_double(dt)), "fm_prepare")


def fm_get_aux(st, what, comp, out):
    p, w = _ptr(out)
    _check(lib().fm_get_aux(st, what, comp, C.c_void_p(p), w), "fm_get_aux")


def fm_residual(st, g, r=None):
    w = _where(list(g) + (list(r) if r is not None else []))
    nrm = C.c_double()
    rv = _vec(r) if r is not None else None
    _check(lib().fm_residual(st, _vec(g), rv, C.byref(nrm), w), "fm_residual")
    return nrm.value


FM_SWEEP_VARIANTS = 36
FM_SWEEP_AUTO = -1
FM_SWEEP_TWO_COLOUR = -2


def fm_smooth(st, e, f, sweeps, variant=FM_SWEEP_AUTO):
    """Smoother row: `sweeps` red-black sweeps on the finest grid; e (list of
    nu float64 arrays) is updated in place."""
    w = _where(list(e) + list(f))
    _check(lib().fm_smooth(st, _vec(e), _vec(f), int(sweeps), int(variant), w), "fm_smooth")


def fm_narrow(inp, out, stream=None):
    """out (float32 CUDA tensor) = inp (float64 CUDA tensor) narrowed as the
    residual kernels narrow the float32 right-hand side."""
    _check(lib().fm_narrow(C.c_void_p(inp.data_ptr()), C.c_void_p(out.data_ptr()), inp.numel(),
                           C.c_void_p(stream)), "fm_narrow")


def fm_wait_selftest(complete, limit_us, stream=None):
    """Status (FM_OK or FM_ETIMEOUT) of the smoother's bounded mbarrier wait
    on a barrier that is completed (complete=True) or that nothing completes."""
    return lib().fm_wait_selftest(1 if complete else 0, int(limit_us), C.c_void_p(stream))


def fm_grid_barrier_selftest(complete, limit_us, stream=None):
    """Status (FM_OK or FM_ETIMEOUT) of the cooperative sweep's bounded grid
    barrier wait, on a count every block reaches (complete=True) or one that
    nothing reaches."""
    return lib().fm_grid_barrier_selftest(1 if complete else 0, int(limit_us), C.c_void_p(stream))


def fm_widen(inp, out, stream=None):
    """out (float64 CUDA tensor) = inp (float32 CUDA tensor) widened as the
    float64 update widens the float32 correction."""
    _check(lib().fm_widen(C.c_void_p(inp.data_ptr()), C.c_void_p(out.data_ptr()), inp.numel(),
                          C.c_void_p(stream)), "fm_widen")


def fm_convolve(st, rho, out):
    w = _where([rho, out])
    _check(lib().fm_convolve(st, C.c_void_p(_ptr(rho)[0]), C.c_void_p(_ptr(out)[0]), w), "fm_convolve")


def fm_restrict(st, fine, coarse):
    w = _where([fine, coarse])
    _check(lib().fm_restrict(st, C.c_void_p(_ptr(fine)[0]), C.c_void_p(_ptr(coarse)[0]), w), "fm_restrict")


def fm_prolong_add(st, coarse, fine):
    w = _where([fine, coarse])
    _check(lib().fm_prolong_add(st, C.c_void_p(_ptr(coarse)[0]), C.c_void_p(_ptr(fine)[0]), w),
           "fm_prolong_add")


def fm_levels(st):
    return lib().fm_levels(st)


def fm_create_batch(grids, prm: fm_params, fn: fm_functional):
    arr = (fm_grid * len(grids))(*grids)
    h = C.c_void_p()
    _check(lib().fm_create_batch(len(grids), arr, C.byref(prm), C.byref(fn), C.byref(h)), "fm_create_batch")
    return h


def fm_destroy_batch(b):
    lib().fm_destroy_batch(b)


def fm_batch_set_stream(b, stream_handle: int):
    _check(lib().fm_batch_set_stream(b, C.c_void_p(stream_handle)), "fm_batch_set_stream")


def fm_batch_instance(b, i):
    return C.c_void_p(lib().fm_batch_instance(b, i))


def fm_step_batch(b, dts):
    n = len(dts)
    arr = (C.c_double * n)(*dts)
    info = (fm_step_info * n)()
    code = lib().fm_step_batch(b, arr, info)
    return code, list(info)


def fm_batch_launches(b):
    return lib().fm_batch_launches(b)


def fm_batch_tuning(b, level):
    v = C.c_int()
    ms = (C.c_float * FM_SWEEP_VARIANTS)()
    _check(lib().fm_batch_tuning(b, level, C.byref(v), ms), "fm_batch_tuning")
    return v.value, list(ms)


def fm_batch_time_smoother(b, iters):
    """(ms per launch, finest points per launch)."""
    ms, pts = C.c_double(), C.c_longlong()
    _check(lib().fm_batch_time_smoother(b, iters, C.byref(ms), C.byref(pts)), "fm_batch_time_smoother")
    return ms.value, pts.value


def fm_batch_time_sweep_variant(b, variant, iters):
    """(ms per launch of fused-sweep variant `variant`, finest points per launch)."""
    ms, pts = C.c_double(), C.c_longlong()
    _check(lib().fm_batch_time_sweep_variant(b, variant, iters, C.byref(ms), C.byref(pts)),
           "fm_batch_time_sweep_variant")
    return ms.value, pts.value


def fm_mass_noalloc(rho, h, out, stream=0):
    """Mass of a float64 CUDA tensor into a 1-element float64 CUDA tensor,
    without any device allocation by the library (see include/fm.h).

    rho must be a contiguous float64 CUDA tensor with 2 or 3 dimensions and
    out a float64 CUDA tensor with at least one element; anything else raises
    ValueError before the C call (the kernel reads rho and writes out as
    device float64 arrays)."""
    import torch
    for name, t in (("rho", rho), ("out", out)):
        if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float64:
            raise ValueError(f"{name} must be a float64 CUDA tensor")
    if rho.dim() not in (2, 3) or not rho.is_contiguous():
        raise ValueError("rho must be a contiguous 2-D or 3-D tensor")
    if out.numel() < 1:
        raise ValueError("out must hold at least one element")
    dims = list(reversed(rho.shape))
    n = (C.c_int * 3)(*(dims + [1] * (3 - len(dims))))
    code = lib().fm_mass_noalloc(C.c_void_p(rho.data_ptr()), len(dims), n, C.c_double(h),
                                 C.c_void_p(out.data_ptr()), C.c_void_p(stream))
    _check(code, "fm_mass_noalloc")


def fm_tuning(st, level):
    """(chosen variant, [ms of every variant]) of the fused sweep at `level`."""
    v = C.c_int()
    ms = (C.c_float * FM_SWEEP_VARIANTS)()
    _check(lib().fm_tuning(st, level, C.byref(v), ms), "fm_tuning")
    return v.value, list(ms)


def fm_profile(st, enable):
    _check(lib().fm_profile(st, 1 if enable else 0), "fm_profile")


def fm_profile_read(st):
    """(smoother_ms, smoother_launches, total_launches)."""
    ms, n, tot = C.c_double(), C.c_longlong(), C.c_longlong()
    _check(lib().fm_profile_read(st, C.byref(ms), C.byref(n), C.byref(tot)), "fm_profile_read")
    return ms.value, n.value, tot.value


class Batch:
    """Independent 2-D instances stepped together (owns an fm_batch)."""

    def __init__(self, kind, sizes, h, alpha=0.0, nu=0.0, precision=FM_FP64, stream=None, **params):
        grids = []
        for n in sizes:
            g = fm_grid()
            g.dim = 2
            ns = list(n) if hasattr(n, "__len__") else [n, n]
            g.n[0], g.n[1], g.n[2] = ns[0], ns[1], 1
            g.h = h
            grids.append(g)
        f = fm_functional()
        f.kind = {"pfc": FM_PFC, "cdft": FM_CDFT}.get(kind, kind)
        f.alpha = alpha
        f.nu = nu
        p = fm_default_params()
        p.precision = precision
        for k, v in params.items():
            setattr(p, k, v)
        self.shapes = [tuple(reversed(list(n) if hasattr(n, "__len__") else [n, n])) for n in sizes]
        self.handle = fm_create_batch(grids, p, f)
        if stream is not None:
            fm_batch_set_stream(self.handle, stream)

    def instance(self, i):
        return fm_batch_instance(self.handle, i)

    def set_fields(self, i, rho, vel):
        fm_set_fields(self.instance(i), rho, vel)

    def get_fields(self, i):
        rho = np.empty(self.shapes[i])
        vel = [np.empty(self.shapes[i]) for _ in range(2)]
        fm_get_fields(self.instance(i), rho, vel)
        return rho, vel

    def step(self, dts):
        code, info = fm_step_batch(self.handle, dts)
        _check(code, "fm_step_batch")
        return info

    def close(self):
        if self.handle:
            fm_destroy_batch(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------------------
# A small object wrapper over the same calls.
# ---------------------------------------------------------------------------
class Solver:
    """One periodic grid and its FAS solver (owns an fm_state handle)."""

    def __init__(self, kind, n, h, dim=2, alpha=0.0, nu=0.0, precision=FM_FP64, stream=None, **params):
        g = fm_grid()
        g.dim = dim
        ns = list(n) if hasattr(n, "__len__") else [n] * dim
        for d in range(3):
            g.n[d] = ns[d] if d < dim else 1
        g.h = h
        f = fm_functional()
        f.kind = {"pfc": FM_PFC, "cdft": FM_CDFT}.get(kind, kind)
        f.alpha = alpha
        f.nu = nu
        p = fm_default_params()
        p.precision = precision
        for k, v in params.items():
            if k == "u_wall":
                p.u_wall[0], p.u_wall[1] = v
            else:
                setattr(p, k, v)
        self.dim = dim
        self.shape = tuple(reversed(ns[:dim]))
        self.model = p.model
        if p.model == FM_GRADFLOW:
            self.nu = 3 if f.kind == FM_PFC else 1
        else:
            self.nu = 1 + dim + (2 if f.kind == FM_PFC else 0)
        self.handle = fm_create(g, p, f)
        if stream is not None:
            fm_set_stream(self.handle, stream)

    def close(self):
        if self.handle:
            fm_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_fields(self, rho, vel):
        fm_set_fields(self.handle, rho, vel)

    def get_fields(self, rho=None, vel=None):
        if rho is None:
            rho = np.empty(self.shape)
            vel = [np.empty(self.shape) for _ in range(self.dim)]
        fm_get_fields(self.handle, rho, vel)
        return rho, vel

    def step(self, dt):
        return fm_step(self.handle, dt)

    def step_host(self, dt, rho_in, vel_in, rho_out, vel_out):
        """One step of host-resident fields (fm_step_host); raises on failure."""
        for a in [rho_in, *vel_in, rho_out, *vel_out]:
            if _ptr(a)[1] != FM_HOST:
                raise ValueError("fm_step_host takes host arrays")
        code, info = fm_step_host(self.handle, dt, rho_in, vel_in, rho_out, vel_out)
        _check(code, "fm_step_host")
        return info

    def host_stepper(self, rho_in, vel_in, rho_out, vel_out):
        """fm_step_host on fixed host buffers, checked and marshalled once:
        the returned callable takes dt and makes one C call per step."""
        return HostStepper(self, rho_in, vel_in, rho_out, vel_out)

    def energy(self):
        return fm_energy(self.handle)

    def mass(self):
        return fm_mass(self.handle)

    def energy_terms(self):
        return fm_energy_terms(self.handle)

    def aux(self, what, comp):
        out = np.empty(self.shape)
        fm_get_aux(self.handle, what, comp, out)
        return out
