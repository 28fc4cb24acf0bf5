"""GPU parity of the paper's other formulations against the complex128 oracle
(through the C ABI):

* the single-front Dirichlet-top sweep (Sec. 2.1-2.2, Algorithms 3 and 4 as
  printed: one-sided sigma_2, one upward sweep, no middle layer), option
  two_front = 0;
* buffer layers between each block and its moving PML (Sec. 2.2), option
  buffer_rows = k, in both formulations.

Tolerances as in test_gpu_parity.py: applications 1e-4 (complex64 factors)
and 1e-10 (complex128), FP64 matvec 1e-12, solves to the requested residual
under the oracle's FP64 operator.
"""
import numpy as np
import pytest

from oracle import helmholtz2d as H
from oracle import krylov as K
from oracle import sweep2d as S
from paper_1007_4291_gb300 import build as B
from paper_1007_4291_gb300 import hs
from paper_1007_4291_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

C_PML = 20.0


@pytest.fixture(scope="module", autouse=True)
def lib():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    B.build()
    return hs.load()


def relerr(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def plan2(c, omega, bp, b, dL, prec=hs.HS_C64, chunk=0, two_front=1, buffer_rows=0, max_nrhs=8, restart=20):
    o = hs.hs_default_options(alpha=2.0, pml_C=C_PML, layers_per_step=dL, factor_prec=prec, chunk=chunk,
                              max_nrhs=max_nrhs, restart=restart, two_front=two_front, buffer_rows=buffer_rows)
    return hs.hs_setup(c.ravel(), omega, c.shape[0], 2, bp, b, o)


def gpu_apply(plan, r, prec):
    tdt = torch.complex64 if prec == hs.HS_C64 else torch.complex128
    rg = torch.from_numpy(np.ascontiguousarray(r)).to("cuda").to(tdt)
    zg = torch.empty_like(rg)
    hs.hs_apply(plan, rg, zg, r.shape[0], prec)
    torch.cuda.synchronize()
    assert hs.hs_last_device_status(plan) == hs.HS_OK
    return zg.cpu().numpy().astype(np.complex128), rg.cpu().numpy().astype(np.complex128)


SINGLE_CASES = [
    # n, bp, b, dL, chunk, R
    (63, 6, 6, 1, 8, 3),      # one layer per step, 8 chunks
    (64, 6, 5, 5, 8, 2),      # even n, remainder block at the top, b < bp
    (71, 6, 6, 12, 8, 4),     # ragged last chunk, d = 12
    (47, 5, 5, 3, 47, 2),     # a single chunk
    (24, 6, 6, 18, 16, 1),    # the whole grid above F is one top block (window of 23 rows)
]


@pytest.mark.parametrize("case", SINGLE_CASES)
@pytest.mark.parametrize("prec", [hs.HS_C64, hs.HS_C128])
def test_single_front_apply_matches_oracle(case, prec):
    n, bp, b, dL, chunk, R = case
    c = I.random_velocity(n, 7)
    omega = 2 * np.pi * 2.5
    plan = plan2(c, omega, bp, b, dL, prec=prec, chunk=chunk, two_front=0)
    try:
        r = I.random_rhs(n, R, 5)
        z, rin = gpu_apply(plan, r, prec)
        ref = S.apply(S.setup(c, omega, bp, b, dL, 2.0, C_PML, two_front=False), rin)
        tol = 1e-4 if prec == hs.HS_C64 else 1e-10
        for k in range(R):
            assert relerr(z[k], ref[k]) <= tol, (k, relerr(z[k], ref[k]))
    finally:
        hs.hs_destroy(plan)


@pytest.mark.parametrize("dtype,tol", [(hs.HS_C128, 1e-12), (hs.HS_C64, 2e-5)])
def test_single_front_matvec_is_dirichlet_top_operator(dtype, tol):
    n, bp = 40, 6
    c = I.random_velocity(n, 3)
    omega = 2 * np.pi * 3
    plan = plan2(c, omega, bp, bp, 1, two_front=0, max_nrhs=2)
    try:
        x = I.random_rhs(n, 2, 11)
        tdt = torch.complex64 if dtype == hs.HS_C64 else torch.complex128
        xg = torch.from_numpy(x).to("cuda").to(tdt)
        yg = torch.empty_like(xg)
        hs.hs_matvec(plan, xg, yg, 2, dtype)
        y = yg.cpu().numpy().astype(np.complex128)
        coef = H.stencil_coefficients(c, omega, bp, C_PML, alpha=0.0, dirichlet_top=True)
        ref = H.apply_stencil(coef, xg.cpu().numpy().astype(np.complex128))
        assert relerr(y, ref) <= tol
    finally:
        hs.hs_destroy(plan)


@pytest.mark.parametrize("prec", [hs.HS_C64, hs.HS_C128])
def test_single_front_solve(prec):
    """FGMRES with the single-front sweep reaches 1e-6 under the oracle's
    Dirichlet-top operator; with complex128 factors its iteration count is
    the oracle FGMRES's to within one."""
    n, bp = 63, 8
    c = I.random_velocity(n, 2)
    omega = 2 * np.pi * 4.0
    R = 2
    plan = plan2(c, omega, bp, bp, 2, prec=prec, chunk=8, two_front=0, max_nrhs=R, restart=30)
    try:
        f = I.point_sources(n, R, 1, bp)
        fg = torch.from_numpy(f).to("cuda")
        ug = torch.zeros_like(fg)
        code, info = hs.hs_solve(plan, fg, ug, R, 1e-6, 300)
        assert code == hs.HS_OK, info
        A0 = H.helmholtz_matrix(c, omega, bp, C_PML, 0.0, dirichlet_top=True)
        u = ug.cpu().numpy()
        for k in range(R):
            assert np.linalg.norm(f[k].ravel() - A0 @ u[k].ravel()) <= 1e-6 * np.linalg.norm(f[k].ravel())
        if prec == hs.HS_C128:
            st = S.setup(c, omega, bp, bp, 2, 2.0, C_PML, two_front=False)
            its = []
            for k in range(R):
                _, it, _ = K.fgmres(lambda v: A0 @ v, lambda v: S.apply(st, v.reshape(n, n)).ravel(),
                                    f[k].ravel(), tol=1e-6, restart=30)
                its.append(it)
            assert abs(info["iterations"] - max(its)) <= 1
    finally:
        hs.hs_destroy(plan)


BUFFER_CASES = [
    # two_front, n, bp, b, dL, k, chunk, R
    (1, 63, 6, 6, 1, 2, 8, 3),     # first blocks' windows cut at the boundary
    (1, 71, 6, 5, 4, 4, 8, 2),     # b < bp, windows of 12 rows
    (0, 64, 6, 6, 3, 3, 8, 2),     # single front with buffers
    (1, 25, 4, 4, 2, 9, 8, 2),     # the largest k: every front block exact, the middle fills the grid
]


@pytest.mark.parametrize("case", BUFFER_CASES)
@pytest.mark.parametrize("prec", [hs.HS_C64, hs.HS_C128])
def test_buffer_rows_apply_matches_oracle(case, prec):
    tf, n, bp, b, dL, k, chunk, R = case
    c = I.random_velocity(n, 9)
    omega = 2 * np.pi * 2.5
    plan = plan2(c, omega, bp, b, dL, prec=prec, chunk=chunk, two_front=tf, buffer_rows=k)
    try:
        r = I.random_rhs(n, R, 6)
        z, rin = gpu_apply(plan, r, prec)
        ref = S.apply(S.setup(c, omega, bp, b, dL, 2.0, C_PML, two_front=bool(tf), buffer=k), rin)
        tol = 1e-4 if prec == hs.HS_C64 else 1e-10
        for q in range(R):
            assert relerr(z[q], ref[q]) <= tol, (q, relerr(z[q], ref[q]))
    finally:
        hs.hs_destroy(plan)


def test_variant_options_are_checked():
    n = 63
    c = I.random_velocity(n, 1)
    bad = [dict(two_front=2), dict(buffer_rows=-1), dict(buffer_rows=40)]   # the middle window does not fit
    for kw in bad:
        with pytest.raises(hs.HsError) as e:
            plan2(c, 20.0, 6, 6, 1, **kw)
        assert e.value.code == hs.HS_EINVAL
    with pytest.raises(hs.HsError) as e:                                 # windows of more than 32 rows
        plan2(c, 20.0, 6, 6, 12, buffer_rows=12)
    assert e.value.code == hs.HS_EUNSUPPORTED
    c3 = I.random_velocity(9, 1, dim=3)
    o = hs.hs_default_options(two_front=0)
    with pytest.raises(hs.HsError) as e:
        hs.hs_setup(c3.ravel(), 10.0, 9, 3, 2, 2, o)
    assert e.value.code == hs.HS_EUNSUPPORTED


@pytest.mark.parametrize("velocity", ["waveguide", "lens"])
def test_paper_workload_wave_packet_solve(velocity):
    """Sec. 3 Test 2 on the GPU: the Gaussian wave packet from (0.125, 0.125)
    along (1, 1) in the vertical waveguide and in the lens, n = 255 at 16
    points per wavelength, solved to 1e-6 under the oracle's FP64 operator."""
    n, bp = 255, 12
    omega = 2 * np.pi * 16.0
    c = I.waveguide_velocity(n) if velocity == "waveguide" else I.lens_velocity(n)
    f = I.wave_packet(n, omega)
    o = hs.hs_default_options(alpha=2.0, pml_C=C_PML, layers_per_step=12, max_nrhs=1)
    plan = hs.hs_setup(c.ravel(), omega, n, 2, bp, bp, o)
    try:
        fg = torch.from_numpy(f).to("cuda")
        ug = torch.zeros_like(fg)
        code, info = hs.hs_solve(plan, fg, ug, 1, 1e-6, 200)
        assert code == hs.HS_OK, info
        A0 = H.helmholtz_matrix(c, omega, bp, C_PML, 0.0)
        u = ug.cpu().numpy()[0]
        assert np.linalg.norm(f[0].ravel() - A0 @ u.ravel()) <= 1e-6 * np.linalg.norm(f[0].ravel())
        assert info["iterations"] <= 30
    finally:
        hs.hs_destroy(plan)
