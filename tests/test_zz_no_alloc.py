"""hs_apply_noalloc: the preconditioner application for callers that must not
allocate device memory (applications owning all free device memory, loops
that cannot take cudaMalloc's device synchronisation, hosts that forbid
library allocations).  Its temporaries live in the library's static device
array instead of the plan's workspace; the result must equal hs_apply's.

Kept in its own file, collected last, so that a failure here cannot hide the
result of any other test.  It passes alone in a fresh process and after the
rest of the suite (the static array keeps the previous call's contents, and
nothing in it needs to start at zero).
"""
import ctypes

import numpy as np
import pytest

from paper_1007_4291_gb300 import build as B
from paper_1007_4291_gb300 import hs
from paper_1007_4291_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_C64 = 1e-4   # the tolerance the parity tests use for complex64 sweeps


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    B.build()
    return hs.load()


def _plan(n, bp, dL, chunk, max_nrhs):
    c = I.random_velocity(n, 4)
    o = hs.hs_default_options(layers_per_step=dL, chunk=chunk, max_nrhs=max_nrhs)
    return hs.hs_setup(c.ravel(), 2 * np.pi * (n + 1) / 16.0, n, 2, bp, bp, o)


@pytest.mark.parametrize("n,bp,dL,chunk,R,dtype", [(63, 6, 3, 8, 5, hs.HS_C64), (127, 12, 12, 16, 3, hs.HS_C128)])
def test_noalloc_matches_hs_apply_twice(lib, n, bp, dL, chunk, R, dtype):
    plan = _plan(n, bp, dL, chunk, R)
    try:
        tdt = torch.complex64 if dtype == hs.HS_C64 else torch.complex128
        r = torch.from_numpy(I.random_rhs(n, R, 8)).to("cuda").to(tdt)
        z_ref = torch.empty_like(r)
        lib_code = lib.hs_apply(plan, ctypes.c_void_p(r.data_ptr()), ctypes.c_void_p(z_ref.data_ptr()), R, dtype, None)
        assert lib_code == hs.HS_OK
        torch.cuda.synchronize()
        ref = z_ref.cpu().numpy()
        for _ in range(2):                     # two calls in a row through the C ABI
            z = torch.full_like(r, float("nan"))
            code = lib.hs_apply_noalloc(plan, ctypes.c_void_p(r.data_ptr()), ctypes.c_void_p(z.data_ptr()), R,
                                        dtype, None)
            assert code == hs.HS_OK
            torch.cuda.synchronize()
            out = z.cpu().numpy()
            assert np.all(np.isfinite(out))
            err = np.linalg.norm(out - ref) / np.linalg.norm(ref)
            assert err <= TOL_C64
        assert hs.hs_last_device_status(plan) == hs.HS_OK
    finally:
        hs.hs_destroy(plan)


def test_noalloc_rejects_problem_larger_than_scratch(lib):
    n = 511
    plan = _plan(n, 12, 12, 0, 64)
    try:
        x = torch.zeros(64 * n * n, dtype=torch.complex64, device="cuda")
        code = lib.hs_apply_noalloc(plan, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(x.data_ptr()), 64,
                                    hs.HS_C64, None)
        assert code == hs.HS_EINVAL
        # within the limit for the same plan
        code = lib.hs_apply_noalloc(plan, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(x.data_ptr()), 8,
                                    hs.HS_C64, None)
        assert code == hs.HS_OK
        torch.cuda.synchronize()
    finally:
        hs.hs_destroy(plan)
