"""Pins of the buffer layers of Sec. 2.2 in the oracle: the moving PML of a
block placed k rows away from it, so that its window is the block rows, k
undamped buffer rows and the b-row PML.  None of these tests uses the CUDA
path.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import helmholtz2d as H
from oracle import sweep2d as S
from paper_1007_4291_gb300 import inputs as I


def test_buffer_window_hand_computed():
    """n = 47 (h = 1/48), b_p = 6, b = 4, d = 2, k = 2.  The lower block of
    rows 9..10 gets the window 4..10 with its Dirichlet row at 3; its damped
    rows are 4, 5, 6 with sigma h / C = 9/64, 4/64, 1/64 (distance 1, 2, 3
    from row 3, width 4 rows) and rows 7..10 (two buffer rows and the block)
    are undamped.  The upper mirror block 38..39 gets 38..44 with rows 42, 43,
    44 damped by 1/64, 4/64, 9/64."""
    n, bp, b, dL, k, C = 47, 6, 4, 2, 2, 20.0
    h = 1.0 / (n + 1)
    om = 2 * np.pi * 3.0
    lower, upper, mid = S.partition(n, bp, b, dL, buffer=k)
    lo, up = lower[2], upper[2]
    assert (lo.lo, lo.hi, lo.wlo, lo.whi, lo.exact) == (9, 10, 4, 10, False)
    assert (up.lo, up.hi, up.wlo, up.whi, up.exact) == (38, 39, 38, 44, False)
    assert (mid.wlo, mid.whi) == (24 - 2 - 4 + 1, 24 + 2 + 4 - 1)
    for blk, sig64 in ((lo, [9, 4, 1, 0, 0, 0, 0]), (up, [0, 0, 0, 0, 1, 4, 9])):
        s_int = S.window_x2_stretch(blk, n, bp, b, C, om)[0]
        want = 1.0 / (1.0 + 1j * (C / h) * np.array(sig64) / 64.0 / om)
        np.testing.assert_allclose(s_int, want, rtol=1e-13)
    # the first lower block (rows 7..8) would need rows from 7 - 2 - 4 + 1 = 2:
    # it fits; with k = 4 it would start at 0, so it is cut at row 1
    first = S.partition(n, bp, b, dL, buffer=4)[0][1]
    assert (first.wlo, first.exact) == (1, True)


@pytest.mark.parametrize("n,bp,dL", [(31, 4, 3), (33, 4, 5)])
def test_buffer_cut_windows_are_exact(n, bp, dL):
    """With the largest k the middle layer allows, k = (n+1)/2 - b, every
    front block's window is cut at the boundary and keeps the operator's
    profile: each T~_B is then the exact Schur inverse (the buffer analogue
    of T4)."""
    c = I.random_velocity(n, 3)
    om, al, C = 2 * np.pi * 3.0, 2.0, 20.0
    k = (n + 1) // 2 - bp
    lower, upper, _ = S.partition(n, bp, bp, dL, buffer=k)
    assert all(B.exact for B in lower[1:] + upper[1:])
    # the middle layer keeps its moving PMLs (its window ends one row short
    # of the boundary on each side), so compare the fronts' blocks
    ex = S.setup(c, om, bp, bp, dL, al, C, full_window=True)
    bf = S.setup(c, om, bp, bp, dL, al, C, buffer=k)
    g = I.random_rhs(n, 1, 4)[0]
    for fe, fb in zip(ex.lower[1:] + ex.upper[1:], bf.lower[1:] + bf.upper[1:]):
        rows = slice(fe.blk.lo - 1, fe.blk.hi)
        a, bb = fe.t_tilde(g[None, rows, :]), fb.t_tilde(g[None, rows, :])
        assert np.linalg.norm(a - bb) <= 1e-10 * np.linalg.norm(a)


def test_single_front_full_buffer_is_exact_inverse():
    """Single front, k beyond the grid: every window reaches x2 = 0, so the
    whole sweep is exact (no middle layer there)."""
    n, bp, dL = 31, 4, 3
    c = I.random_velocity(n, 5)
    om, al, C = 2 * np.pi * 3.0, 2.0, 20.0
    A = H.helmholtz_matrix(c, om, bp, C, al, dirichlet_top=True)
    f = I.random_rhs(n, 1, 9)[0]
    st = S.setup(c, om, bp, bp, dL, al, C, two_front=False, buffer=n)
    ref = spla.spsolve(A.tocsc(), f.ravel())
    assert np.linalg.norm(S.apply(st, f).ravel() - ref) <= 1e-10 * np.linalg.norm(ref)


def test_buffer_improves_half_space_approximation():
    """Sec. 2.2: a buffer makes T~_m a better approximation of the half-space
    T_m (constant velocity, b = 4): the relative error falls as k = 0, 2, 4."""
    n, bp, al, C, b = 95, 12, 2.0, 20.0, 4
    om = 2 * np.pi * (n + 1) / 16.0
    c = I.constant_velocity(n)
    A = H.helmholtz_matrix(c, om, bp, C, al).tocsc()
    m = (n + 1) // 2 - 4
    x = np.arange(1, n + 1) / (n + 1)
    g = np.exp(-((x - 0.5) / 0.05) ** 2).astype(np.complex128)
    lu = spla.splu(A[: m * n, : m * n].tocsc())
    rhs = np.zeros(m * n, dtype=np.complex128)
    rhs[(m - 1) * n:] = g
    exact = lu.solve(rhs)[(m - 1) * n:]
    errs = []
    for k in (0, 2, 4):
        blk = S._lower_window(m, m, b, k, False)
        t = S.factor_block(blk, c, om, bp, b, C, al).t_tilde(g.reshape(1, 1, n))[0, 0]
        errs.append(np.linalg.norm(t - exact) / np.linalg.norm(exact))
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 0.5 * errs[0]
