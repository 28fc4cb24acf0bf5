"""CPU-side checks of the C ABI: the library builds, loads, exports every
function declared in include/hs.h, and rejects invalid arguments before any
device work.  No compute call is made here."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_1007_4291_gb300 import build as B
from paper_1007_4291_gb300 import hs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return hs.load()


def declared_functions():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names += re.findall(r"\b(hs_[a-z0-9_]+)\s*\(", txt)
    return sorted(set(names))


def test_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert "hs_setup" in names and "hs_apply" in names and "hs_matvec" in names and "hs_solve" in names
    for name in names:
        assert hasattr(lib, name), name
    assert set(hs.EXPORTED) <= set(names)


def test_default_options_and_strerror(lib):
    o = hs.hs_default_options()
    assert o.alpha == 2.0 and o.layers_per_step == 12 and o.factor_prec == hs.HS_C64
    for code in range(8):
        assert len(hs.strerror(code)) > 3


@pytest.mark.parametrize("n,bp,b,err", [(32, 4, 4, hs.HS_EINVAL),     # even n
                                        (9, 5, 5, hs.HS_EINVAL),      # 2 bp + 1 > n
                                        (31, 4, 6, hs.HS_EINVAL),     # b > bp + 1
                                        (31, 4, 0, hs.HS_EINVAL)])
def test_setup_rejects_invalid_sizes(lib, n, bp, b, err):
    c = np.ones(n * n)
    plan = ctypes.c_void_p()
    o = hs.hs_default_options()
    code = lib.hs_setup(c.ctypes.data, 10.0, n, 2, bp, b, ctypes.byref(o), None, ctypes.byref(plan))
    assert code == err and not plan.value


def test_setup_rejects_bad_velocity_and_options(lib):
    n = 15
    plan = ctypes.c_void_p()
    c = np.ones(n * n)
    c[7] = -1.0
    o = hs.hs_default_options()
    assert lib.hs_setup(c.ctypes.data, 10.0, n, 2, 3, 3, ctypes.byref(o), None, ctypes.byref(plan)) == hs.HS_EINVAL
    c[7] = np.nan
    assert lib.hs_setup(c.ctypes.data, 10.0, n, 2, 3, 3, ctypes.byref(o), None, ctypes.byref(plan)) == hs.HS_EINVAL
    c[:] = 1.0
    o.factor_prec = 32
    assert lib.hs_setup(c.ctypes.data, 10.0, n, 2, 3, 3, ctypes.byref(o), None, ctypes.byref(plan)) == hs.HS_EINVAL
    o = hs.hs_default_options(sep_rhs_per_cta=3)          # 1, 2 or 4 RHS per separator-solve CTA (or 0)
    assert lib.hs_setup(c.ctypes.data, 10.0, n, 2, 3, 3, ctypes.byref(o), None, ctypes.byref(plan)) == hs.HS_EINVAL
    o = hs.hs_default_options(async_setup=2)               # 0 or 1
    assert lib.hs_setup(c.ctypes.data, 10.0, n, 2, 3, 3, ctypes.byref(o), None, ctypes.byref(plan)) == hs.HS_EINVAL
    assert hs.hs_default_options().async_setup == 0
    o = hs.hs_default_options()
    assert lib.hs_setup(c.ctypes.data, 10.0, n, 4, 3, 3, ctypes.byref(o), None, ctypes.byref(plan)) == hs.HS_EINVAL
    # 3D: sizes are checked before the n^3 velocities are read
    assert lib.hs_setup(c.ctypes.data, 10.0, 257, 3, 3, 3, ctypes.byref(o), None, ctypes.byref(plan)) == hs.HS_EUNSUPPORTED
    # 2D: point indices are 32-bit, checked before the n^2 velocities are read
    assert lib.hs_setup(c.ctypes.data, 10.0, 32769, 2, 3, 3, ctypes.byref(o), None, ctypes.byref(plan)) == hs.HS_EUNSUPPORTED
    c3 = np.ones(7 ** 3)
    c3[100] = 0.0
    assert lib.hs_setup(c3.ctypes.data, 10.0, 7, 3, 2, 2, ctypes.byref(o), None, ctypes.byref(plan)) == hs.HS_EINVAL
    assert lib.hs_setup(None, 10.0, n, 2, 3, 3, ctypes.byref(o), None, ctypes.byref(plan)) == hs.HS_EINVAL
    # batched setup with options per problem: one factor precision for all, options required
    cs = (ctypes.c_void_p * 2)(c.ctypes.data, c.ctypes.data)
    om = (ctypes.c_double * 2)(10.0, 10.0)
    nn = (ctypes.c_int * 2)(n, n)
    outs = (ctypes.c_void_p * 2)()
    oa = (hs.HsOptions * 2)(hs.hs_default_options(), hs.hs_default_options(factor_prec=hs.HS_C128))
    assert lib.hs_setup_batched_opts(2, cs, om, nn, 2, 3, 3, oa, None, outs) == hs.HS_EINVAL
    assert lib.hs_setup_batched_opts(2, cs, om, nn, 2, 3, 3, None, None, outs) == hs.HS_EINVAL
    assert not outs[0] and not outs[1]
    assert lib.hs_apply(None, None, None, 1, 64, None) == hs.HS_EINVAL
    assert lib.hs_destroy(None) == hs.HS_OK
