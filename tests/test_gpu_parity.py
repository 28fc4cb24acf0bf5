"""GPU parity of libhs against the complex128 oracle (through the C ABI).

Tolerances: FP64 paths 1e-12 (matvec) / 1e-10 (sweep, chained block
solves); complex64 factors and sweeps 1e-4 relative L2 (the stated bar for
preconditioner applications); solutions must reach the requested relative
residual when their residual is recomputed by the oracle's FP64 operator.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import helmholtz2d as H
from oracle import sweep2d as S
from paper_1007_4291_gb300 import build as B
from paper_1007_4291_gb300 import hs
from paper_1007_4291_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

C_PML = 20.0
C_MOVING = None      # library default: the moving PMLs take the boundary C (Eq. helma reuses sigma_2)


@pytest.fixture(scope="module", autouse=True)
def lib():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    B.build()
    return hs.load()


def relerr(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def make_plan(c, omega, bp, b, dL, prec=hs.HS_C64, chunk=0, alpha=2.0, max_nrhs=8, restart=20, Cm=None):
    n = c.shape[0]
    o = hs.hs_default_options(alpha=alpha, pml_C=C_PML, layers_per_step=dL, factor_prec=prec, chunk=chunk,
                              max_nrhs=max_nrhs, restart=restart, moving_pml_C=Cm or 0.0)
    return hs.hs_setup(c.ravel(), omega, n, 2, bp, b, o)


def gpu(x, dtype=torch.complex128):
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda").to(dtype)


def run_apply(plan, r, dtype):
    tdt = torch.complex64 if dtype == hs.HS_C64 else torch.complex128
    rg = gpu(r, tdt)
    zg = torch.empty_like(rg)
    hs.hs_apply(plan, rg, zg, r.shape[0], dtype)
    torch.cuda.synchronize()
    assert hs.hs_last_device_status(plan) == hs.HS_OK
    return zg.cpu().numpy().astype(np.complex128)


# ---------------------------------------------------------------- A2 matvec

@pytest.mark.parametrize("n", [31, 65])
@pytest.mark.parametrize("dtype,tol", [(hs.HS_C128, 1e-12), (hs.HS_C64, 2e-5)])
def test_matvec_matches_oracle(n, dtype, tol):
    c = I.random_velocity(n, 3)
    omega, bp = 2 * np.pi * 3, 6
    plan = make_plan(c, omega, bp, bp, 1)
    try:
        x = I.random_rhs(n, 3, 11)
        tdt = torch.complex64 if dtype == hs.HS_C64 else torch.complex128
        xg = gpu(x, tdt)
        yg = torch.empty_like(xg)
        hs.hs_matvec(plan, xg, yg, 3, dtype)
        y = yg.cpu().numpy().astype(np.complex128)
        coef = H.stencil_coefficients(c, omega, bp, C_PML, alpha=0.0)
        xin = x.astype(np.complex64).astype(np.complex128) if dtype == hs.HS_C64 else x
        ref = H.apply_stencil(coef, xin)
        assert relerr(y, ref) <= tol
    finally:
        hs.hs_destroy(plan)


@pytest.mark.parametrize("n,bp,C", [(31, 15, C_PML),   # PML-free square of one point
                                    (33, 4, 0.0),      # no damping: the square is the whole grid
                                    (35, 3, C_PML)])
@pytest.mark.parametrize("dtype,tol", [(hs.HS_C128, 1e-12), (hs.HS_C64, 2e-5)])
def test_matvec_square_and_band_split(n, bp, C, dtype, tol):
    """The matvec runs the PML-free square and the PML band as two kernels;
    every point is covered once whatever the square's size."""
    c = I.random_velocity(n, 4)
    omega = 2 * np.pi * 2
    o = hs.hs_default_options(pml_C=C, layers_per_step=1, max_nrhs=2)
    plan = hs.hs_setup(c.ravel(), omega, n, 2, bp, bp, o)
    try:
        x = I.random_rhs(n, 2, 12)
        tdt = torch.complex64 if dtype == hs.HS_C64 else torch.complex128
        xg = gpu(x, tdt)
        yg = torch.full_like(xg, float("nan"))
        hs.hs_matvec(plan, xg, yg, 2, dtype)
        y = yg.cpu().numpy().astype(np.complex128)
        assert np.isfinite(y).all()
        coef = H.stencil_coefficients(c, omega, bp, C, alpha=0.0)
        xin = x.astype(np.complex64).astype(np.complex128) if dtype == hs.HS_C64 else x
        assert relerr(y, H.apply_stencil(coef, xin)) <= tol
    finally:
        hs.hs_destroy(plan)


# ---------------------------------------------------------------- A3-A6 apply

APPLY_CASES = [
    # n, bp, b, dL, chunk, nrhs
    (63, 6, 6, 1, 8, 5),      # 8 chunks, d = 1 (one layer per step)
    (63, 6, 6, 3, 8, 3),      # d = 3, remainder block
    (71, 6, 5, 5, 8, 4),      # ragged last chunk (71 = 8*8 + 7), b < bp
    (63, 6, 6, 4, 63, 2),     # a single chunk: no separators
    (45, 5, 5, 2, 2, 1),      # minimum chunk length, one RHS
    (13, 6, 6, 3, 4, 2),      # n = 2 bp + 1: no lower/upper blocks, F, E and the middle only
    (41, 4, 4, 20, 6, 3),     # d larger than a front: one remainder block per front
    (31, 5, 5, 2, 16, 2),     # two chunks: one separator (twist only)
    (47, 5, 5, 3, 16, 2),     # three chunks: twist with a top chain and no bottom chain
    (79, 6, 6, 4, 8, 3),      # ten chunks: both half chains
]


@pytest.mark.parametrize("case", APPLY_CASES)
@pytest.mark.parametrize("prec,Cm", [(hs.HS_C64, None), (hs.HS_C128, None), (hs.HS_C64, 2 * C_PML)])
def test_apply_matches_oracle(case, prec, Cm):
    """Cm None: the paper's single constant (library default); 2C: the opt-in
    separate moving-PML strength."""
    n, bp, b, dL, chunk, R = case
    c = I.random_velocity(n, 7)
    omega, alpha = 2 * np.pi * 2.5, 2.0
    plan = make_plan(c, omega, bp, b, dL, prec=prec, chunk=chunk, alpha=alpha, Cm=Cm)
    try:
        r = I.random_rhs(n, R, 5)
        st = S.setup(c, omega, bp, b, dL, alpha, C_PML, Cm=Cm)
        io = hs.HS_C64 if prec == hs.HS_C64 else hs.HS_C128
        rin = r.astype(np.complex64).astype(np.complex128) if io == hs.HS_C64 else r
        ref = S.apply(st, rin)
        z = run_apply(plan, r, io)
        tol = 1e-4 if prec == hs.HS_C64 else 1e-10
        for k in range(R):
            assert relerr(z[k], ref[k]) <= tol, (k, relerr(z[k], ref[k]))
    finally:
        hs.hs_destroy(plan)


def test_apply_c128_io_with_c64_factors_and_alias():
    """dtype selects the I/O type only; r and z may alias."""
    n, bp = 39, 5
    c = I.lens_velocity(n)
    omega = 2 * np.pi * 2.0
    plan = make_plan(c, omega, bp, bp, 2, chunk=6)
    try:
        r = I.random_rhs(n, 2, 1)
        ref = S.apply(S.setup(c, omega, bp, bp, 2, 2.0, C_PML, Cm=C_MOVING), r)
        rg = gpu(r)
        hs.hs_apply(plan, rg, rg, 2, hs.HS_C128)
        assert relerr(rg.cpu().numpy(), ref) <= 1e-4
    finally:
        hs.hs_destroy(plan)


def test_apply_rejects_bad_nrhs():
    n = 15
    plan = make_plan(I.constant_velocity(n), 20.0, 3, 3, 1, max_nrhs=2)
    try:
        x = torch.zeros(3 * n * n, dtype=torch.complex64, device="cuda")
        with pytest.raises(hs.HsError):
            hs.hs_apply(plan, x, x, 3, hs.HS_C64)
        with pytest.raises(hs.HsError):
            hs.hs_apply(plan, x, x, 0, hs.HS_C64)
    finally:
        hs.hs_destroy(plan)


# ---------------------------------------------------------------- A7 solve

@pytest.mark.parametrize("prec", [hs.HS_C64, hs.HS_C128])
def test_solve_reaches_tolerance_under_oracle_operator(prec):
    n, bp = 63, 8
    c = I.random_velocity(n, 2)
    omega = 2 * np.pi * 4.0
    R = 4
    plan = make_plan(c, omega, bp, bp, 1, prec=prec, chunk=16, max_nrhs=R, restart=10)
    try:
        f = I.point_sources(n, R, 1, bp)
        fg = gpu(f)
        ug = torch.zeros_like(fg)
        code, info = hs.hs_solve(plan, fg, ug, R, 1e-6, 200)
        assert code == hs.HS_OK, info
        u = ug.cpu().numpy()
        A0 = H.helmholtz_matrix(c, omega, bp, C_PML, 0.0)
        for k in range(R):
            res = np.linalg.norm(f[k].ravel() - A0 @ u[k].ravel()) / np.linalg.norm(f[k].ravel())
            assert res <= 1e-6
            ref = spla.spsolve(A0.tocsc(), f[k].ravel())
            assert relerr(u[k].ravel(), ref) <= 1e-4
        assert info["iterations"] <= 40
    finally:
        hs.hs_destroy(plan)


def test_solve_iteration_count_matches_oracle():
    """The GPU FGMRES (c128 factors) and the oracle FGMRES need the same
    number of iterations within one on the same problem."""
    from oracle import krylov as K
    n, bp = 47, 6
    c = I.random_velocity(n, 9)
    omega = 2 * np.pi * 3.0
    plan = make_plan(c, omega, bp, bp, 2, prec=hs.HS_C128, chunk=8, max_nrhs=1, restart=30)
    try:
        f = I.point_sources(n, 1, 4, bp)
        fg = gpu(f)
        ug = torch.zeros_like(fg)
        code, info = hs.hs_solve(plan, fg, ug, 1, 1e-8, 100)
        assert code == hs.HS_OK
        A0 = H.helmholtz_matrix(c, omega, bp, C_PML, 0.0)
        st = S.setup(c, omega, bp, bp, 2, 2.0, C_PML, Cm=C_MOVING)
        _, it, _ = K.fgmres(lambda v: A0 @ v, lambda v: S.apply(st, v.reshape(n, n)).ravel(), f[0].ravel(),
                            tol=1e-8, restart=30)
        assert abs(info["iterations"] - it) <= 1
    finally:
        hs.hs_destroy(plan)


def test_solve_with_c64_factors_reaches_fp64_class_tolerance():
    """The complex64 path keeps its Krylov vectors in double-float (48-bit
    significand): it must reach a 1e-10 relative residual, measured by the
    oracle's FP64 operator, which single precision cannot represent."""
    n, bp = 47, 6
    c = I.random_velocity(n, 12)
    omega = 2 * np.pi * 3.0
    R = 3
    plan = make_plan(c, omega, bp, bp, 2, prec=hs.HS_C64, chunk=8, max_nrhs=R, restart=20)
    try:
        f = I.point_sources(n, R, 6, bp)
        fg = gpu(f)
        ug = torch.zeros_like(fg)
        code, info = hs.hs_solve(plan, fg, ug, R, 1e-10, 300)
        assert code == hs.HS_OK, info
        A0 = H.helmholtz_matrix(c, omega, bp, C_PML, 0.0)
        u = ug.cpu().numpy()
        for k in range(R):
            res = np.linalg.norm(f[k].ravel() - A0 @ u[k].ravel()) / np.linalg.norm(f[k].ravel())
            assert res <= 1e-10, res
    finally:
        hs.hs_destroy(plan)


@pytest.mark.parametrize("tol", [1e-6, 1e-10])
def test_refinement_mode_reaches_tolerance(tol):
    """FP32-basis FGMRES cycles restarted from the double-float residual
    (krylov_basis = 1) reach FP64-class tolerances under the oracle's operator."""
    n, bp = 63, 8
    c = I.random_velocity(n, 2)
    omega = 2 * np.pi * 4.0
    R = 3
    o = hs.hs_default_options(alpha=2.0, pml_C=C_PML, layers_per_step=1, chunk=16, max_nrhs=R, restart=20,
                              krylov_basis=1, inner_tol=1e-5)
    plan = hs.hs_setup(c.ravel(), omega, n, 2, bp, bp, o)
    try:
        f = I.point_sources(n, R, 1, bp)
        fg = gpu(f)
        ug = torch.zeros_like(fg)
        code, info = hs.hs_solve(plan, fg, ug, R, tol, 300)
        assert code == hs.HS_OK, info
        A0 = H.helmholtz_matrix(c, omega, bp, C_PML, 0.0)
        u = ug.cpu().numpy()
        for k in range(R):
            res = np.linalg.norm(f[k].ravel() - A0 @ u[k].ravel()) / np.linalg.norm(f[k].ravel())
            assert res <= tol, res
        print("refinement to %g: %d iterations in %d cycles" % (tol, info["iterations"], info["restarts"]))
    finally:
        hs.hs_destroy(plan)
