"""The allocation-free mass entry point (fm_mass_noalloc), for callers that
cannot call cudaMalloc, agrees with the allocating fm_mass of an fm_state.

Collected last on purpose: if it fails, a run that stops at the first failure
has already run every other test.  Two calls in a row check that the scratch
left behind by one call does not leak into the next."""
import numpy as np
import pytest

from paper_1503_07416_gb300 import fm

pytestmark = pytest.mark.gpu


def test_mass_noalloc_matches_fm_mass_twice():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1503_07416_gb300 import build
    build.build_library()
    stream = torch.cuda.current_stream().cuda_stream
    rng = np.random.default_rng(99)
    for shape, h in (((96, 128), 0.7), ((40, 24), 0.9)):
        rho = 0.8 + 0.1 * rng.uniform(-1, 1, shape)
        sol = fm.Solver("pfc", list(reversed(shape)), h, alpha=0.6, stream=stream)
        sol.set_fields(rho, [np.zeros(shape), np.zeros(shape)])
        ref = sol.mass()
        sol.close()
        dev = torch.from_numpy(rho).cuda()
        out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        fm.fm_mass_noalloc(dev, h, out, stream)
        torch.cuda.synchronize()
        got = float(out.item())
        assert abs(got - ref) <= 1e-13 * abs(ref), (got, ref)
    # sizes beyond the scratch maximum are rejected
    big = torch.empty(1, dtype=torch.float64, device="cuda")
    n = (fm.C.c_int * 3)(4096, 1025, 1)
    code = fm.lib().fm_mass_noalloc(fm.C.c_void_p(big.data_ptr()), 2, n, fm.C.c_double(1.0),
                                    fm.C.c_void_p(out.data_ptr()), fm.C.c_void_p(stream))
    assert code == fm.FM_EINVAL
