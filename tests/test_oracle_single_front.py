"""Pins of the single-front, Dirichlet-top formulation in the oracle (Sec.
2.1-2.2, Algorithms 3 and 4 as printed: PML at x2 = 0 only through the
one-sided sigma_2 of Eq. sigma, zero Dirichlet values at x2 = 1, one upward
sweep from the front F, no middle layer).  None of these tests uses the CUDA
path.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import helmholtz2d as H
from oracle import krylov as K
from oracle import sweep2d as S
from paper_1007_4291_gb300 import inputs as I


def test_one_sided_profile_closed_form():
    """sigma_2 of Eq. sigma: C/eta at x2 = 0, C/(4 eta) at eta/2, zero from
    eta on, in particular at and near x2 = 1."""
    C, eta = 20.0, 0.1
    t = np.array([0.0, eta / 2, eta, 0.5, 1 - eta / 2, 1.0])
    np.testing.assert_allclose(H.pml_sigma_one_sided(t, eta, C), [C / eta, C / (4 * eta), 0, 0, 0, 0], atol=1e-12)


def test_dirichlet_top_operator_rows():
    """The Dirichlet-top operator equals the all-sides one on the lower half
    of the grid, and near x2 = 1 its x2 couplings are unstretched:
    N h^2 s1(ih) = 1.  It stays complex symmetric."""
    n, bp = 31, 5
    c = I.random_velocity(n, 3)
    om = 2 * np.pi * 3.0
    top = H.stencil_coefficients(c, om, bp, 20.0, 2.0, dirichlet_top=True)
    both = H.stencil_coefficients(c, om, bp, 20.0, 2.0)
    half = (n - 1) // 2
    for k in ("E", "W", "N", "S", "D"):
        np.testing.assert_array_equal(top[k][:half], both[k][:half])
    assert not np.allclose(top["N"][-bp:], both["N"][-bp:])
    h = 1.0 / (n + 1)
    s1 = H.axis_stretch(n, bp, 20.0, om)[0][1:n + 1]
    np.testing.assert_allclose(top["N"][-bp:] * h**2 * s1[None, :], 1.0, rtol=1e-14)
    A = H.helmholtz_matrix(c, om, bp, 20.0, 2.0, dirichlet_top=True).toarray()
    assert np.abs(A - A.T).max() <= 1e-15 * np.abs(A).max()


def test_single_partition_covers_rows_once():
    for n, bp, dL in [(127, 12, 1), (127, 12, 12), (2047, 12, 12), (64, 6, 5)]:
        blocks, upper, mid = S.partition_single(n, bp, bp, dL)
        assert upper == [] and mid is None
        rows = np.concatenate([B.rows for B in blocks])
        assert rows.tolist() == list(range(1, n + 1))
        assert blocks[0].kind == "F" and blocks[-1].hi == n
        assert all(B.wlo >= 1 and B.whi <= n and B.whi == B.hi for B in blocks)


@pytest.mark.parametrize("n,bp,dL", [(15, 3, 1), (31, 4, 3), (33, 4, 5), (24, 4, 2)])
def test_T3_single_front_exact_sweep_reproduces_direct_solve(n, bp, dL):
    """Algorithms 1 + 2 in the single-front order invert A_alpha exactly."""
    c = I.random_velocity(n, 10 + n)
    om, al, C = 2 * np.pi * 2.5, 1.0, 20.0
    A = H.helmholtz_matrix(c, om, bp, C, al, dirichlet_top=True)
    f = I.random_rhs(n, 1, 7)[0]
    ref = spla.spsolve(A.tocsc(), f.ravel())
    ex = S.exact_setup_single(c, om, bp, bp, dL, al, C)
    u = S.exact_apply_single(ex, f).ravel()
    assert np.linalg.norm(u - ref) <= 1e-10 * np.linalg.norm(ref)


@pytest.mark.parametrize("n,bp,dL", [(15, 3, 1), (31, 4, 3), (33, 4, 5)])
def test_T4_single_front_full_window_is_exact_inverse(n, bp, dL):
    """With windows down to x2 = 0, every T~_B is the exact Schur inverse, so
    Algorithm 4 with one front applies A_alpha^{-1}: pins the partition, the
    couplings and the top block's missing backward step."""
    c = I.random_velocity(n, 3)
    om, al, C = 2 * np.pi * 3.0, 2.0, 20.0
    A = H.helmholtz_matrix(c, om, bp, C, al, dirichlet_top=True)
    f = I.random_rhs(n, 2, 9)
    st = S.setup(c, om, bp, bp, dL, al, C, full_window=True, two_front=False)
    u = S.apply(st, f)
    for r in range(2):
        ref = spla.spsolve(A.tocsc(), f[r].ravel())
        assert np.linalg.norm(u[r].ravel() - ref) <= 1e-10 * np.linalg.norm(ref)


def test_T4_planted_two_sided_profile_fails(monkeypatch):
    """Planted mistake: the sweep's F block built with the all-sides profile
    while the operator is Dirichlet-top.  With full windows the mismatch in
    the x2 stretch of the windows breaks exactness."""
    n, bp, dL = 31, 4, 3
    c = I.random_velocity(n, 3)
    om, al, C = 2 * np.pi * 3.0, 2.0, 20.0
    A = H.helmholtz_matrix(c, om, bp, C, al, dirichlet_top=True)
    f = I.random_rhs(n, 1, 9)[0]
    monkeypatch.setattr(H, "pml_sigma_one_sided", H.pml_sigma)
    st = S.setup(c, om, bp, bp, dL, al, C, full_window=True, two_front=False)
    ref = spla.spsolve(A.tocsc(), f.ravel())
    assert np.linalg.norm(S.apply(st, f).ravel() - ref) > 1e-6 * np.linalg.norm(ref)


def test_single_front_preconditions():
    """Behaviour: the single-front moving-PML sweep makes FGMRES converge on
    the Dirichlet-top problem (lens field, n = 127, 16 points per wavelength)
    in far fewer iterations than without a preconditioner."""
    n, bp = 127, 12
    c = I.lens_velocity(n)
    om = 2 * np.pi * 8.0
    A0 = H.helmholtz_matrix(c, om, bp, 20.0, 0.0, dirichlet_top=True)
    f = I.centered_source(n)[0].ravel()
    st = S.setup(c, om, bp, bp, 12, 2.0, 20.0, two_front=False)
    P = lambda v: S.apply(st, v.reshape(n, n)).ravel()
    x, it, _ = K.fgmres(lambda v: A0 @ v, P, f, tol=1e-6, restart=30)
    assert np.linalg.norm(f - A0 @ x) <= 1e-6 * np.linalg.norm(f)
    assert it <= 20
