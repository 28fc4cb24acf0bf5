"""hs_apply_noalloc: the preconditioner application for callers that must not
allocate device memory (applications owning all free device memory, loops
that cannot take cudaMalloc's device synchronisation, hosts that forbid
library allocations).  Its temporaries live in the library's static device
array instead of the plan's workspace, and it runs the same kernels with the
same launch shapes as hs_apply, so its result must equal hs_apply's bit for
bit.

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


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    B.build()
    return hs.load()


def _plan(n, bp, dL, chunk, max_nrhs, prec):
    c = I.random_velocity(n, 4)
    o = hs.hs_default_options(layers_per_step=dL, chunk=chunk, max_nrhs=max_nrhs, factor_prec=prec)
    return hs.hs_setup(c.ravel(), 2 * np.pi * (n + 1) / 16.0, n, 2, bp, bp, o)


def _call(lib, fn, plan, r, z, R, dtype):
    return getattr(lib, fn)(plan, ctypes.c_void_p(r.data_ptr()), ctypes.c_void_p(z.data_ptr()), R, dtype, None)


@pytest.mark.parametrize("n,bp,dL,chunk,R,prec", [(63, 6, 3, 8, 5, hs.HS_C64), (127, 12, 12, 16, 3, hs.HS_C128)])
def test_noalloc_matches_hs_apply_twice(lib, n, bp, dL, chunk, R, prec):
    plan = _plan(n, bp, dL, chunk, R, prec)
    try:
        tdt = torch.complex64 if prec == hs.HS_C64 else torch.complex128
        r = torch.from_numpy(I.random_rhs(n, R, 8)).to("cuda").to(tdt)
        z_ref = torch.empty_like(r)
        assert _call(lib, "hs_apply", plan, r, z_ref, R, prec) == hs.HS_OK
        torch.cuda.synchronize()
        ref = z_ref.cpu().numpy()
        assert np.all(np.isfinite(ref))
        for _ in range(2):                     # two calls in a row through the C ABI
            z = torch.full_like(r, float("nan"))
            assert _call(lib, "hs_apply_noalloc", plan, r, z, R, prec) == hs.HS_OK
            torch.cuda.synchronize()
            out = z.cpu().numpy()
            assert np.array_equal(out, ref)    # same kernels and launch shapes: identical bits
        # the plan's own workspace is untouched: hs_apply after it still agrees
        z2 = torch.empty_like(r)
        assert _call(lib, "hs_apply", plan, r, z2, R, prec) == hs.HS_OK
        torch.cuda.synchronize()
        assert np.array_equal(z2.cpu().numpy(), ref)
        assert hs.hs_last_device_status(plan) == hs.HS_OK
    finally:
        hs.hs_destroy(plan)


def test_noalloc_rejects_sizes_beyond_its_limits(lib):
    n = 511
    plan = _plan(n, 12, 12, 0, 64, hs.HS_C64)
    try:
        x = torch.zeros(65 * n * n, dtype=torch.complex64, device="cuda")
        # larger than the 32 MiB static scratch
        assert _call(lib, "hs_apply_noalloc", plan, x, x, 64, hs.HS_C64) == hs.HS_EINVAL
        # more right-hand sides than the plan was set up for
        assert _call(lib, "hs_apply_noalloc", plan, x, x, 65, hs.HS_C64) == hs.HS_EINVAL
        assert _call(lib, "hs_apply_noalloc", plan, x, x, 0, hs.HS_C64) == hs.HS_EINVAL
        # within the limits for the same plan
        assert _call(lib, "hs_apply_noalloc", plan, x, x, 8, hs.HS_C64) == hs.HS_OK
        torch.cuda.synchronize()
    finally:
        hs.hs_destroy(plan)
