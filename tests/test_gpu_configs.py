"""Parity on the configured 2D workloads (GPU), against the oracle.

* Plain FP64 method: n = 127, omega/2pi = 8, b_p = b = 12, one grid line per
  layer, constant c = 1, one Gaussian source (s = h) at the centre,
  complex128 factors, GMRES to 1e-6.  The application equals the oracle's
  M_alpha to 1e-10; the solution reaches 1e-6 under the oracle's FP64
  operator, matches a sparse direct solve, and takes the oracle FGMRES's
  iteration count within one.
* n = 511, omega/2pi = 32, 64 point sources, complex64 factors, d = 12, on
  the smooth random field and on the converging lens: a sampled RHS of the
  application equals the oracle's to 1e-4; all 64 solutions reach 1e-6 under
  the oracle's FP64 operator.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import helmholtz2d as H
from oracle import krylov as K
from oracle import sweep2d as S
from paper_1007_4291_gb300 import build as B
from paper_1007_4291_gb300 import hs
from paper_1007_4291_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

C_PML = 20.0
C_MOVING = None      # library default: the moving PMLs take the boundary C (Eq. helma reuses sigma_2)
ALPHA = 2.0


@pytest.fixture(scope="module", autouse=True)
def lib():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    B.build()
    return hs.load()


def relerr(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def test_plain_fp64_method_n127():
    n, bp, dL = 127, 12, 1
    omega = 2 * np.pi * 8.0
    c = I.constant_velocity(n)
    f = I.centered_source(n)
    o = hs.hs_default_options(alpha=ALPHA, pml_C=C_PML, layers_per_step=dL, factor_prec=hs.HS_C128,
                              max_nrhs=1, restart=30)
    plan = hs.hs_setup(c.ravel(), omega, n, 2, bp, bp, o)
    try:
        st = S.setup(c, omega, bp, bp, dL, ALPHA, C_PML, Cm=C_MOVING)
        fg = torch.from_numpy(f).to("cuda")
        zg = torch.empty_like(fg)
        hs.hs_apply(plan, fg, zg, 1, hs.HS_C128)
        assert relerr(zg.cpu().numpy()[0], S.apply(st, f[0])) <= 1e-10

        ug = torch.zeros_like(fg)
        code, info = hs.hs_solve(plan, fg, ug, 1, 1e-6, 200)
        assert code == hs.HS_OK, info
        u = ug.cpu().numpy()[0].ravel()
        A0 = H.helmholtz_matrix(c, omega, bp, C_PML, 0.0)
        assert np.linalg.norm(f[0].ravel() - A0 @ u) / np.linalg.norm(f[0].ravel()) <= 1e-6
        assert relerr(u, spla.spsolve(A0.tocsc(), f[0].ravel())) <= 1e-4
        _, it, _ = K.fgmres(lambda v: A0 @ v, lambda v: S.apply(st, v.reshape(n, n)).ravel(), f[0].ravel(),
                            tol=1e-6, restart=30)
        print("n = 127 plain FP64 method: GPU %d iterations, oracle %d" % (info["iterations"], it))
        assert abs(info["iterations"] - it) <= 1
    finally:
        hs.hs_destroy(plan)


@pytest.mark.parametrize("field", ["random", "lens"])
def test_n511_complex64_64_rhs(field):
    n, bp, dL, R = 511, 12, 12, 64
    omega = 2 * np.pi * 32.0
    c = I.random_velocity(n, 0) if field == "random" else I.lens_velocity(n)
    o = hs.hs_default_options(alpha=ALPHA, pml_C=C_PML, layers_per_step=dL, max_nrhs=R)
    plan = hs.hs_setup(c.ravel(), omega, n, 2, bp, bp, o)
    try:
        f = I.point_sources(n, R, 3, bp)
        fg = torch.from_numpy(f).to("cuda")
        zg = torch.empty_like(fg)
        hs.hs_apply(plan, fg, zg, R, hs.HS_C128)
        st = S.setup(c, omega, bp, bp, dL, ALPHA, C_PML, Cm=C_MOVING)
        k = 41                                      # one sampled RHS
        assert relerr(zg[k].cpu().numpy(), S.apply(st, f[k])) <= 1e-4

        ug = torch.zeros_like(fg)
        code, info = hs.hs_solve(plan, fg, ug, R, 1e-6, 400)
        assert code == hs.HS_OK, info
        A0 = H.helmholtz_matrix(c, omega, bp, C_PML, 0.0)
        u = ug.cpu().numpy()
        res = [np.linalg.norm(f[q].ravel() - A0 @ u[q].ravel()) / np.linalg.norm(f[q].ravel()) for q in range(R)]
        print("n = 511 %s field, 64 RHS: %d iterations, max true residual %.2e" % (field, info["iterations"],
                                                                                   max(res)))
        assert max(res) <= 1e-6
    finally:
        hs.hs_destroy(plan)
