"""Parity at the headline size, in the launch configuration bench.py times
(n = 2047, omega/2pi = 128, b_p = b = 12, d = 12, alpha = 2, complex64
factors, default chunking, 64 RHS).

* One RHS of the sweep application against the oracle's M_alpha (LAPACK band
  solves of all 173 subproblems; about a minute on the host): 1e-4.
* The 64-RHS FGMRES solve: every solution's true relative residual, computed
  by the oracle's sparse FP64 operator on the host, is below 1e-6.
"""
import numpy as np
import pytest

from oracle import helmholtz2d as H
from oracle import sweep2d as S
from paper_1007_4291_gb300 import build as B
from paper_1007_4291_gb300 import hs
from paper_1007_4291_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

N, R, BP, DL, ALPHA, C = 2047, 64, 12, 12, 2.0, 20.0
OMEGA = 2 * np.pi * (N + 1) / 16.0


@pytest.fixture(scope="module")
def plan():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    B.build()
    c = I.random_velocity(N, 0)
    o = hs.hs_default_options(alpha=ALPHA, pml_C=C, layers_per_step=DL, max_nrhs=R)
    p = hs.hs_setup(c.ravel(), OMEGA, N, 2, BP, BP, o)
    yield c, o, p
    hs.hs_destroy(p)


def test_fullsize_sweep_application_matches_oracle(plan):
    c, o, p = plan
    r = I.random_rhs(N, R, 1)
    rg = torch.from_numpy(r).to("cuda").to(torch.complex64)
    zg = torch.empty_like(rg)
    hs.hs_apply(p, rg, zg, R, hs.HS_C64)
    assert hs.hs_sync(p) == hs.HS_OK
    k = 17                                           # one sampled RHS
    z = zg[k].cpu().numpy().astype(np.complex128)
    st = S.setup(c, OMEGA, BP, BP, DL, ALPHA, C, Cm=o.moving_pml_C or None)
    ref = S.apply(st, rg[k].cpu().numpy().astype(np.complex128))
    err = float(np.linalg.norm(z - ref) / np.linalg.norm(ref))
    print("n = 2047 sweep application, RHS %d: relative error %.2e" % (k, err))
    assert err <= 1e-4


def test_fullsize_solve_residuals_under_oracle_operator(plan):
    c, o, p = plan
    f = I.point_sources(N, R, 1, BP)
    fg = torch.from_numpy(f).to("cuda")
    ug = torch.zeros_like(fg)
    code, info = hs.hs_solve(p, fg, ug, R, 1e-6, 400)
    assert code == hs.HS_OK, info
    A0 = H.helmholtz_matrix(c, OMEGA, BP, C, 0.0)
    u = ug.cpu().numpy()
    res = [np.linalg.norm(f[k].ravel() - A0 @ u[k].ravel()) / np.linalg.norm(f[k].ravel()) for k in range(R)]
    print("n = 2047, 64 RHS: %d iterations, max true residual %.2e" % (info["iterations"], max(res)))
    assert max(res) <= 1e-6
