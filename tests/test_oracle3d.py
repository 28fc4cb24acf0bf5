"""Pins of the 3D oracle (CPU only): symmetry, the textbook 7-point operator
at C = 0, exact Schur-complement sweeps and full-window sweeps against a
sparse direct solve, and the free-space Green's function of a point source."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle import helmholtz3d as H3
from oracle import sweep2d as S2
from paper_1007_4291_gb300 import inputs as I


def test_operator_is_complex_symmetric():
    n = 7
    c = I.random_velocity(n, 1, dim=3)
    A = H3.helmholtz_matrix(c, 2 * np.pi * 1.5, 2, 10.0, alpha=1.0)
    d = abs(A - A.T).max()
    assert d <= 1e-15 * abs(A).max()


def test_zero_pml_is_textbook_laplacian_plus_mass():
    n, omega, alpha = 6 + 1, 9.0, 0.7
    c = I.random_velocity(n, 2, dim=3)
    A = H3.helmholtz_matrix(c, omega, 2, 0.0, alpha=alpha)
    h = 1.0 / (n + 1)
    T = sp.diags([np.ones(n - 1), -2 * np.ones(n), np.ones(n - 1)], [-1, 0, 1]) / h ** 2
    Id = sp.identity(n)
    L = sp.kron(sp.kron(Id, Id), T) + sp.kron(sp.kron(Id, T), Id) + sp.kron(sp.kron(T, Id), Id)
    M = sp.diags(((omega + 1j * alpha) ** 2 / c ** 2).ravel())
    assert abs(A - (L + M)).max() <= 1e-9 * abs(A).max()


@pytest.mark.parametrize("n,dL", [(7, 1), (9, 2)])
def test_exact_schur_sweep_reproduces_direct_solve(n, dL):
    c = I.random_velocity(n, 3, dim=3)
    omega, alpha, C, bp, b = 2 * np.pi * 1.5, 1.0, 10.0, 2, 2
    f = I.random_rhs(n, 1, 4, dim=3)[0]
    u = H3.exact_apply(c, omega, bp, b, dL, alpha, C, f)
    A = H3.helmholtz_matrix(c, omega, bp, C, alpha).tocsc()
    ref = spla.spsolve(A, f.ravel()).reshape(n, n, n)
    assert np.linalg.norm(u - ref) <= 1e-10 * np.linalg.norm(ref)


@pytest.mark.parametrize("n,dL", [(7, 1), (9, 3)])
def test_full_window_sweep_is_exact_inverse(n, dL):
    """With windows reaching the boundary (and the boundary profile) T~_B is
    the exact Schur inverse, so M_alpha = A_alpha^{-1}."""
    c = I.random_velocity(n, 5, dim=3)
    omega, alpha, C, bp, b = 2 * np.pi * 1.5, 1.0, 10.0, 2, 2
    st = H3.setup(c, omega, bp, b, dL, alpha, C, full_window=True)
    f = I.random_rhs(n, 2, 6, dim=3)
    u = H3.apply(st, f)
    A = H3.helmholtz_matrix(c, omega, bp, C, alpha).tocsc()
    for k in range(2):
        ref = spla.spsolve(A, f[k].ravel()).reshape(n, n, n)
        assert np.linalg.norm(u[k] - ref) <= 1e-10 * np.linalg.norm(ref)


def test_stencil_apply_matches_matrix():
    n = 6 + 1
    c = I.random_velocity(n, 7, dim=3)
    coef = H3.coefficients(c, 11.0, 2, 10.0, 0.5)
    x = I.random_rhs(n, 2, 8, dim=3)
    A = H3.assemble(coef)
    y = H3.apply_stencil(coef, x)
    for k in range(2):
        assert np.allclose(y[k].ravel(), A @ x[k].ravel(), rtol=1e-13, atol=1e-9)


def test_moving_pml_sweep_preconditions_well():
    """M_alpha A is close to the identity away from the PML: GMRES on a
    moderate 3D problem converges in few iterations (the paper reports
    11-13 at tolerance 1e-3)."""
    from oracle import krylov as K
    n, bp, b = 15, 4, 4
    c = I.random_velocity(n, 9, dim=3)
    omega = 2 * np.pi * (n + 1) / 8.0
    st = H3.setup(c, omega, bp, b, 1, 1.0, 20.0)
    A = H3.helmholtz_matrix(c, omega, bp, 20.0, 0.0)
    f = I.point_sources(n, 1, 10, bp, dim=3)[0].ravel()
    x, it, _ = K.fgmres(lambda v: A @ v, lambda v: H3.apply(st, v.reshape(n, n, n)).ravel(), f, tol=1e-6,
                        restart=30)
    assert np.linalg.norm(f - A @ x) <= 1e-6 * np.linalg.norm(f)
    assert it <= 20


def test_point_source_matches_green_function():
    """Constant c = 1, alpha = 0: the solution of A u = f for a unit-mass
    Gaussian source approximates -exp(i k r) / (4 pi r) away from the source
    and the PML, with the second-order error of the 7-point scheme."""
    errs = []
    for n in (15, 31):
        omega = 2 * np.pi * 2.0
        bp = (n + 1) // 5
        c = np.ones((n, n, n))
        A = H3.helmholtz_matrix(c, omega, bp, 20.0, 0.0).tocsc()
        h = 1.0 / (n + 1)
        x = h * np.arange(1, n + 1)
        Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
        s = h
        r2 = (X - 0.5) ** 2 + (Y - 0.5) ** 2 + (Z - 0.5) ** 2
        f = np.exp(-r2 / (2 * s * s)) / ((2 * np.pi) ** 1.5 * s ** 3)
        u = spla.spsolve(A, f.ravel()).reshape(n, n, n)
        r = np.sqrt(r2)
        shell = (r >= 0.15) & (r <= 0.28)
        g = -np.exp(1j * omega * r[shell]) / (4 * np.pi * r[shell])
        errs.append(np.linalg.norm(u[shell] - g) / np.linalg.norm(g))
    assert errs[1] <= 0.2
    assert errs[1] <= 0.5 * errs[0]


def test_planted_sign_error_in_x3_coupling_fails_symmetry_pin():
    n = 5
    c = I.random_velocity(n, 11, dim=3)
    coef = H3.coefficients(c, 7.0, 1, 10.0, 0.0)
    coef["U"] = -coef["U"]
    A = H3.assemble(coef)
    assert abs(A - A.T).max() > 1e-6 * abs(A).max()
