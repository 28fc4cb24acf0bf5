"""Pins of the complex128 oracle against facts fixed by the paper and by mathematics.

None of these tests uses the CUDA path.  Each pin is chosen so that a
plausible slip in the oracle (a dropped term, a wrong sign or index, a
transposed operand, a misplaced PML) fails at least one of them; the
``planted`` tests check that claim by patching a mistake into the oracle.
"""
import json
import os

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla
import scipy.special as ss

from oracle import helmholtz2d as H
from oracle import krylov as K
from oracle import sweep2d as S
from paper_1007_4291_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- Eq. sigma

def test_pml_profile_closed_form():
    """Eq. sigma: quadratic ramp C/eta at the boundary, zero at depth eta and
    in the interior, symmetric about 1/2; s = 1 where sigma = 0."""
    C, eta = 20.0, 0.1
    t = np.array([0.0, eta / 2, eta, 0.5, 1 - eta, 1 - eta / 2, 1.0])
    sig = H.pml_sigma(t, eta, C)
    np.testing.assert_allclose(sig, [C / eta, C / (4 * eta), 0, 0, 0, C / (4 * eta), C / eta], atol=1e-12)
    s = H.stretch(sig, 7.0)
    assert s[3] == 1.0
    np.testing.assert_allclose(1 / s[0], 1 + 1j * (C / eta) / 7.0)


# ---------------------------------------------------------------- T1 / T2

def test_T1_complex_symmetric_block_tridiagonal():
    """A = A^t; A_{m,m} tridiagonal; A_{m,m+-1} diagonal; no other blocks."""
    n, bp = 15, 3
    c = I.random_velocity(n, 0)
    A = H.helmholtz_matrix(c, 2 * np.pi * 2.0, bp, 20.0, alpha=1.5).toarray()
    assert np.abs(A - A.T).max() <= 1e-15 * np.abs(A).max()
    for m in range(n):
        for k in range(n):
            blk = A[m * n:(m + 1) * n, k * n:(k + 1) * n]
            if m == k:
                assert np.count_nonzero(np.triu(blk, 2)) == 0 and np.count_nonzero(np.tril(blk, -2)) == 0
                assert np.all(np.diag(blk, 1) != 0)
            elif abs(m - k) == 1:
                assert np.count_nonzero(blk - np.diag(np.diag(blk))) == 0
                assert np.all(np.diag(blk) != 0)
            else:
                assert np.count_nonzero(blk) == 0


def test_T2_textbook_laplacian_when_no_pml():
    """C = 0: A_alpha is the Dirichlet 5-point Laplacian (Kronecker sum) plus
    (omega + i alpha)^2 / c^2 on the diagonal."""
    n = 13
    h = 1.0 / (n + 1)
    c = I.random_velocity(n, 5)
    om, al = 9.0, 1.25
    A = H.helmholtz_matrix(c, om, 3, 0.0, alpha=al)
    T = sp.diags([np.ones(n - 1), -2 * np.ones(n), np.ones(n - 1)], [-1, 0, 1]) / h**2
    L = sp.kron(sp.identity(n), T) + sp.kron(T, sp.identity(n))
    ref = L + sp.diags(((om + 1j * al) ** 2 / c**2).ravel())
    assert abs(A - ref).max() <= 1e-9 * abs(ref).max()


def test_stencil_apply_matches_assembly():
    """Two independent codings of Eq. helmd agree (point stencil vs CSR)."""
    n = 17
    c = I.random_velocity(n, 1)
    coef = H.stencil_coefficients(c, 2 * np.pi * 3, 4, 20.0, alpha=2.0)
    A = H.assemble(coef)
    x = I.random_rhs(n, 3, 2)
    y = H.apply_stencil(coef, x)
    for r in range(3):
        np.testing.assert_allclose(y[r].ravel(), A @ x[r].ravel(), rtol=1e-13, atol=1e-13 * abs(y).max())


# ---------------------------------------------------------------- T3 / T4

@pytest.mark.parametrize("n,bp,dL", [(7, 2, 1), (15, 3, 1), (15, 3, 2), (31, 4, 1), (31, 4, 3), (31, 5, 4)])
def test_T3_exact_sweep_reproduces_direct_solve(n, bp, dL):
    """Algorithms 1 + 2 in the two-front, d-layer block order (Eq. Afact)
    invert A_alpha exactly."""
    c = I.random_velocity(n, 10 + n, lo=0.8, hi=1.2)
    om, al, C = 2 * np.pi * 2.5, 1.0, 20.0
    A = H.helmholtz_matrix(c, om, bp, C, al)
    f = I.random_rhs(n, 1, 7)[0]
    ref = spla.spsolve(A.tocsc(), f.ravel())
    ex = S.exact_setup(c, om, bp, bp, dL, al, C)
    u = S.exact_apply(ex, f).ravel()
    assert np.linalg.norm(u - ref) <= 1e-10 * np.linalg.norm(ref)


@pytest.mark.parametrize("n,bp,dL", [(15, 3, 1), (31, 4, 1), (31, 4, 3), (33, 4, 5)])
def test_T4_full_window_sweep_is_exact_inverse(n, bp, dL):
    """With windows reaching the boundary on the eliminated side, T~_B is the
    (B,B) block of the truncated inverse, which equals S_B^{-1} (Sec. 2.2);
    then Algorithm 4 with two fronts applies A_alpha^{-1} exactly.  Pins the
    partition, the couplings A_{m+1,m}, F/E handling and the middle block."""
    c = I.random_velocity(n, 3)
    om, al, C = 2 * np.pi * 3.0, 2.0, 20.0
    A = H.helmholtz_matrix(c, om, bp, C, al)
    f = I.random_rhs(n, 2, 9)
    st = S.setup(c, om, bp, bp, dL, al, C, full_window=True)
    u = S.apply(st, f)
    for r in range(2):
        ref = spla.spsolve(A.tocsc(), f[r].ravel())
        assert np.linalg.norm(u[r].ravel() - ref) <= 1e-10 * np.linalg.norm(ref)


def test_partition_covers_rows_once():
    for n, bp, dL in [(127, 12, 1), (127, 12, 12), (2047, 12, 12), (511, 12, 5)]:
        lower, upper, mid = S.partition(n, bp, bp, dL)
        rows = np.concatenate([B.rows for B in lower + upper + [mid]])
        assert sorted(rows.tolist()) == list(range(1, n + 1))
        assert lower[-1].hi + 1 == mid.lo and upper[-1].lo - 1 == mid.hi
        assert all(B.wlo >= 1 and B.whi <= n for B in lower + upper + [mid])


# ---------------------------------------------------------------- T6

def _dense_window_matrix(coef):
    """Lexicographic (x1 fastest) dense matrix of a window operator."""
    D = coef["D"]
    w, n = D.shape
    M = np.zeros((w * n, w * n), dtype=np.complex128)
    for j in range(w):
        for i in range(n):
            p = j * n + i
            M[p, p] = D[j, i]
            if i + 1 < n:
                M[p, p + 1] = coef["E"][j, i]
            if i > 0:
                M[p, p - 1] = coef["W"][j, i]
            if j + 1 < w:
                M[p, p + n] = coef["N"][j, i]
            if j > 0:
                M[p, p - n] = coef["S"][j, i]
    return M


@pytest.mark.parametrize("dL", [1, 3])
def test_T6_band_lu_equals_dense_solve(dL):
    """The x2-first band LU (Algorithm 3) solves H_B exactly: compare with a
    dense solve of H_B in the lexicographic ordering, for every block kind."""
    n, bp, b = 21, 4, 4
    c = I.random_velocity(n, 4)
    om, al, C = 2 * np.pi * 2.0, 2.0, 20.0
    lower, upper, mid = S.partition(n, bp, b, dL)
    rng = np.random.default_rng(0)
    for blk in [lower[0], lower[1], upper[0], upper[-1], mid]:
        fb = S.factor_block(blk, c, om, bp, b, C, al)
        coef = S.window_coefficients(blk, c, om, bp, b, C, al)
        M = _dense_window_matrix(coef)
        assert np.abs(M - M.T).max() <= 1e-12 * np.abs(M).max()        # H_B symmetric
        d = blk.hi - blk.lo + 1
        g = rng.standard_normal((2, d, n)) + 1j * rng.standard_normal((2, d, n))
        out = fb.t_tilde(g)
        for r in range(2):
            rhs = np.zeros((blk.w, n), dtype=np.complex128)
            rhs[blk.lo - blk.wlo: blk.lo - blk.wlo + d] = g[r]
            x = np.linalg.solve(M, rhs.ravel()).reshape(blk.w, n)
            ref = x[blk.lo - blk.wlo: blk.lo - blk.wlo + d]
            assert np.linalg.norm(out[r] - ref) <= 1e-11 * np.linalg.norm(ref)


def test_moving_profile_vanishes_on_block_rows():
    """Eq. helma: s2^m = 1 on the block rows, damped below (lower), above
    (upper) or on both sides (middle), strongest next to the Dirichlet row."""
    n, bp, b, dL = 63, 6, 6, 2
    lower, upper, mid = S.partition(n, bp, b, dL)
    for blk in [lower[3], upper[3], mid]:
        s_int, s_up, s_dn = S.window_x2_stretch(blk, n, bp, b, 20.0, 10.0)
        rows = np.arange(blk.wlo, blk.whi + 1)
        inside = (rows >= blk.lo) & (rows <= blk.hi)
        assert np.all(s_int[inside] == 1.0)
        sig = np.imag(1 / s_int)
        if blk.kind in ("lower", "middle"):
            assert sig[0] > sig[1] > 0
        if blk.kind in ("upper", "middle"):
            assert sig[-1] > sig[-2] > 0


# ---------------------------------------------------------------- T5

def _hankel_error(n, C=20.0, freq=4.0, patch=None):
    omega = 2 * np.pi * freq
    bp = (n + 1) // 8
    c = I.constant_velocity(n)
    A = H.helmholtz_matrix(c, omega, bp, C, 0.0)
    f = I.centered_source(n)[0]
    u = spla.spsolve(A.tocsc(), f.ravel()).reshape(n, n)
    h = 1.0 / (n + 1)
    x = h * np.arange(1, n + 1)
    X1, X2 = np.meshgrid(x, x)
    r = np.hypot(X1 - 0.5, X2 - 0.5)
    m = (r >= 0.1) & (r <= 0.3)
    g = -0.25j * ss.hankel1(0, omega * r[m])
    return np.linalg.norm(u[m] - g) / np.linalg.norm(g)


def test_T5_hankel_green_function_second_order():
    """Constant c = 1, unit-mass Gaussian source: u -> -(i/4) H0^(1)(omega r)
    away from the source and the PML, with error falling ~4x per halving of h
    (second-order 5-point scheme; the PML must absorb the outgoing wave)."""
    e = [_hankel_error(n) for n in (63, 127, 255)]
    assert e[2] < 0.01
    assert e[0] / e[1] > 3.3 and e[1] / e[2] > 3.3


def test_T5_planted_wrong_pml_sign_fails(monkeypatch):
    """Planted mistake: stretching with the conjugate (anti-absorbing) factor
    breaks the Hankel pin."""
    monkeypatch.setattr(H, "stretch", lambda sig, om: 1.0 / (1.0 - 1j * np.asarray(sig) / om))
    e = [_hankel_error(n) for n in (63, 127)]
    assert not (e[0] / e[1] > 3.3 and e[1] < 0.02)


# ---------------------------------------------------------------- T7 / behaviour

def test_T7_fgmres_matches_direct_solve():
    n, bp = 31, 5
    c = I.random_velocity(n, 2)
    om = 2 * np.pi * 3.0
    A0 = H.helmholtz_matrix(c, om, bp, 20.0, 0.0)
    f = I.point_sources(n, 1, 1, bp)[0].ravel()
    ref = spla.spsolve(A0.tocsc(), f)
    st = S.setup(c, om, bp, bp, 1, 2.0, 20.0)
    P = lambda v: S.apply(st, v.reshape(n, n)).ravel()
    x, it, hist = K.fgmres(lambda v: A0 @ v, P, f, tol=1e-8, restart=10)
    assert np.linalg.norm(f - A0 @ x) <= 1e-8 * np.linalg.norm(f)
    assert np.linalg.norm(x - ref) <= 1e-5 * np.linalg.norm(ref)
    x2, it2, _ = K.fgmres(lambda v: A0 @ v, lambda v: v, f, tol=1e-8, restart=200, maxit=2000)
    assert np.linalg.norm(x2 - ref) <= 1e-5 * np.linalg.norm(ref)
    assert it < it2                                     # the sweep preconditions
    xl, itl, _ = K.gmres_left(lambda v: A0 @ v, P, f, tol=1e-10)
    assert np.linalg.norm(xl - ref) <= 1e-6 * np.linalg.norm(ref)


def _paper_setting_iterations():
    n, fr = 127, 16.0                       # q = 8 points per wavelength
    omega = 2 * np.pi * fr
    c = I.lens_velocity(n)
    A0 = H.helmholtz_matrix(c, omega, 12, 20.0, 0.0)
    st = S.setup(c, omega, 12, 12, 12, 2.0, 20.0)
    f = I.centered_source(n, center=(0.5, 0.125))[0].ravel()
    P = lambda v: S.apply(st, v.reshape(n, n)).ravel()
    _, it, _ = K.gmres_left(lambda v: A0 @ v, P, f, tol=1e-3, maxit=200)
    return it


def test_behaviour_paper_iteration_band():
    """Sec. 3 settings (q = 8, alpha = 2, b = d = 12, two fronts, tol 1e-3):
    the paper reports 11-26 iterations across its 2D tables; with this
    synthetic lens the count must not exceed the paper's largest."""
    with open(os.path.join(GOLDEN, "paper_2d_iterations.json")) as fh:
        gold = json.load(fh)
    its = [row["n_iter"] for tbl in gold["tables"] for row in tbl["rows"]]
    it = _paper_setting_iterations()
    assert 1 <= it <= max(its)


def test_behaviour_planted_missing_moving_pml(monkeypatch):
    """Planted mistake: without the moving PML (Dirichlet right below each
    block) the same solve needs far more iterations than the paper's band."""
    monkeypatch.setattr(S, "moving_sigma", lambda t, e, C: np.zeros_like(np.asarray(t, dtype=float)))
    assert _paper_setting_iterations() > 26


def test_moving_pml_strength_is_a_preconditioner_parameter():
    """Cm changes only the moving profiles of the subproblems: F, E keep the
    boundary profile (their T~ are exact Schur inverses of A's blocks), and
    Cm = C reproduces the single-constant setup."""
    from paper_1007_4291_gb300 import inputs as I
    n, bp, b, dL = 23, 4, 4, 3
    c = I.random_velocity(n, 3)
    omega = 2 * np.pi * 2.0
    r = I.random_rhs(n, 1, 4)[0]
    base = S.apply(S.setup(c, omega, bp, b, dL, 2.0, 20.0), r)
    same = S.apply(S.setup(c, omega, bp, b, dL, 2.0, 20.0, Cm=20.0), r)
    other = S.apply(S.setup(c, omega, bp, b, dL, 2.0, 20.0, Cm=40.0), r)
    assert np.array_equal(base, same)
    assert not np.allclose(base, other)
    lower, upper, _ = S.partition(n, bp, b, dL)
    for blk in (lower[0], upper[0]):          # F and E
        s1 = S.window_x2_stretch(blk, n, bp, b, 20.0, omega, Cm=40.0)
        s0 = S.window_x2_stretch(blk, n, bp, b, 20.0, omega)
        assert all(np.array_equal(x, y) for x, y in zip(s0, s1))
    moving = lower[1]
    s1 = S.window_x2_stretch(moving, n, bp, b, 20.0, omega, Cm=40.0)[0]
    s0 = S.window_x2_stretch(moving, n, bp, b, 20.0, omega)[0]
    assert not np.allclose(s0, s1) and np.allclose(s0[-dL:], 1.0) and np.allclose(s1[-dL:], 1.0)


# ---------------------------------------------------------------- moving PML (Eq. helma)
#
# Hand-computed values of the moving profile.  Grid n = 47 (h = 1/48), boundary
# PML b_p = 6, moving PML b = 4 != b_p, d = 2 rows per step, C = 20.  Eq. helma
# shifts the one-sided profile of Eq. sigma so that it starts at the row lo - b
# (the window's Dirichlet row) and uses eta = b h, so on the window of a lower
# block [lo..hi] = [9..10] (window rows 6..10) the distance to the Dirichlet
# row 5 is t = 1, 2, 3, 4, 5 grid spacings and
#   sigma = (C / (4h)) ((t - 4)/4)^2 = (C/h) (t - 4)^2 / 64   for t <= 4, else 0.
# The tables below hold sigma h / C in 64ths, worked out by hand, at the window
# rows, at the half points above them (j + 1/2) and below them (j - 1/2).
_HAND = dict(
    n=47, bp=6, b=4, dL=2, C=20.0,
    lower=dict(index=2, rows=(6, 10), lo=9, hi=10,
               at=[9, 4, 1, 0, 0], up=[6.25, 2.25, 0.25, 0, 0], dn=[12.25, 6.25, 2.25, 0.25, 0]),
    # upper block [38..39], window 38..42, Dirichlet row 43 (= hi + b)
    upper=dict(index=2, rows=(38, 42), lo=38, hi=39,
               at=[0, 0, 1, 4, 9], up=[0, 0.25, 2.25, 6.25, 12.25], dn=[0, 0, 0.25, 2.25, 6.25]),
    # middle layer 24, window 21..27, Dirichlet rows 20 and 28: both profiles
    middle=dict(rows=(21, 27), lo=24, hi=24,
                at=[9, 4, 1, 0, 1, 4, 9], up=[6.25, 2.25, 0.25, 0.25, 2.25, 6.25, 12.25],
                dn=[12.25, 6.25, 2.25, 0.25, 0.25, 2.25, 6.25]),
)


def _hand_profile_mismatches(window_stretch, Cm=None):
    """Compare window_stretch (the 2D x2 or the 3D x3 moving stretch) with the
    hand table; returns the list of mismatching (kind, which) pairs."""
    g = _HAND
    n, bp, b, dL, C = g["n"], g["bp"], g["b"], g["dL"], g["C"]
    Cm = C if Cm is None else Cm
    h = 1.0 / (n + 1)
    omega = 2 * np.pi * 3.0
    lower, upper, mid = S.partition(n, bp, b, dL)
    blocks = dict(lower=lower[g["lower"]["index"]], upper=upper[g["upper"]["index"]], middle=mid)
    bad = []
    for kind, blk in blocks.items():
        e = g[kind]
        assert (blk.wlo, blk.whi, blk.lo, blk.hi) == (e["rows"][0], e["rows"][1], e["lo"], e["hi"])
        got = window_stretch(blk, n, bp, b, C, omega, Cm=Cm)
        for which, vals in zip(("at", "up", "dn"), got):
            sig = (Cm / h) * np.array(e[which], dtype=np.float64) / 64.0
            want = 1.0 / (1.0 + 1j * sig / omega)
            if not np.allclose(vals, want, rtol=1e-13, atol=0):
                bad.append((kind, which))
    return bad


def test_moving_profile_hand_computed_values():
    """Eq. helma with b != b_p: s2^m at the window rows and half points of a
    lower, an upper and the middle block equals the hand-computed table (both
    at the paper's single constant C and at another strength), in 2D and for
    the x3 profile of the 3D slabs."""
    from oracle import helmholtz3d as H3
    assert _hand_profile_mismatches(S.window_x2_stretch) == []
    assert _hand_profile_mismatches(S.window_x2_stretch, Cm=40.0) == []
    assert _hand_profile_mismatches(H3.window_x3_stretch) == []


@pytest.mark.parametrize("slip", ["C_not_over_eta", "eta_from_bp", "shift_up", "shift_down"])
def test_moving_profile_planted_slips_fail_hand_pin(monkeypatch, slip):
    """Planted mistakes in the moving profile each break the hand table:
    strength C instead of C/eta_b, eta_b = b_p h instead of b h, and the
    profile shifted by one row either way."""
    orig = S.moving_sigma
    h = 1.0 / (_HAND["n"] + 1)
    planted = {
        "C_not_over_eta": lambda t, e, C: orig(t, e, C) * e,
        "eta_from_bp": lambda t, e, C: orig(t, _HAND["bp"] * h, C),
        "shift_up": lambda t, e, C: orig(np.asarray(t) + h, e, C),
        "shift_down": lambda t, e, C: orig(np.asarray(t) - h, e, C),
    }[slip]
    monkeypatch.setattr(S, "moving_sigma", planted)
    assert _hand_profile_mismatches(S.window_x2_stretch) != []


# Physics of the moving PML (Sec. 2.2): T_m, the (m, m) block of the inverse of
# A_alpha restricted to the half space of rows 1..m (zero Dirichlet values on
# row m + 1), is the discrete half-space Green's function on row m; T~_m
# replaces everything below row m - b + 1 by a PML of b rows.  For constant
# velocity the approximation must improve as b grows and be close at b = 12
# (the paper's width).  The reference T_m is a sparse direct solve of the
# truncated operator, independent of the window and band code.
_GREEN = dict(n=95, bp=12, alpha=2.0, C=20.0, widths=(4, 8, 12), bounds=(5e-3, 4e-4, 1e-4))


def _half_space_errors(kind):
    import scipy.sparse.linalg as spla_
    g = _GREEN
    n, bp, al, C = g["n"], g["bp"], g["alpha"], g["C"]
    omega = 2 * np.pi * (n + 1) / 16.0          # 16 points per wavelength
    c = I.constant_velocity(n)
    A = H.helmholtz_matrix(c, omega, bp, C, al).tocsc()
    h = 1.0 / (n + 1)
    x = h * np.arange(1, n + 1)
    gsrc = np.exp(-((x - 0.5) / 0.05) ** 2).astype(np.complex128)   # smooth load on row m
    m = (n + 1) // 2 - 4 if kind == "lower" else (n + 1) // 2 + 4
    if kind == "lower":
        sub = np.arange(0, m * n)                   # rows 1..m
        pos = slice((m - 1) * n, m * n)
    else:
        sub = np.arange((m - 1) * n, n * n)         # rows m..n
        pos = slice(0, n)
    lu = spla_.splu(A[sub][:, sub].tocsc())
    rhs = np.zeros(sub.size, dtype=np.complex128)
    rhs[pos] = gsrc
    exact = lu.solve(rhs)[pos]
    errs = []
    for b in g["widths"]:
        blk = S.Block(kind, m, m, m - b + 1 if kind == "lower" else m, m if kind == "lower" else m + b - 1)
        approx = S.factor_block(blk, c, omega, bp, b, C, al).t_tilde(gsrc.reshape(1, 1, n))[0, 0]
        errs.append(np.linalg.norm(approx - exact) / np.linalg.norm(exact))
    return errs


def _half_space_pin_holds(errs):
    return all(e < bound for e, bound in zip(errs, _GREEN["bounds"])) and errs[0] > errs[1] > errs[2]


@pytest.mark.parametrize("kind", ["lower", "upper"])
def test_moving_pml_approximates_half_space_green_function(kind):
    """||T~_m g - T_m g|| / ||T_m g|| falls as the moving PML widens
    (b = 4, 8, 12) and is below 1e-4 at b = 12, for both fronts."""
    errs = _half_space_errors(kind)
    assert _half_space_pin_holds(errs), errs


@pytest.mark.parametrize("slip", ["C_not_over_eta", "eta_from_bp", "shift_up", "shift_down"])
def test_moving_pml_planted_slips_fail_green_pin(monkeypatch, slip):
    """The same planted slips of the profile also break the half-space pin."""
    orig = S.moving_sigma
    h = 1.0 / (_GREEN["n"] + 1)
    planted = {
        "C_not_over_eta": lambda t, e, C: orig(t, e, C) * e,
        "eta_from_bp": lambda t, e, C: orig(t, _GREEN["bp"] * h, C),
        "shift_up": lambda t, e, C: orig(np.asarray(t) + h, e, C),
        "shift_down": lambda t, e, C: orig(np.asarray(t) - h, e, C),
    }[slip]
    monkeypatch.setattr(S, "moving_sigma", planted)
    assert not _half_space_pin_holds(_half_space_errors("lower"))


@pytest.mark.parametrize("velocity,table", [("lens", "2DPML1"), ("waveguide", "2DPML2"), ("random", "2DPML3")])
@pytest.mark.parametrize("test", [1, 2])
def test_behaviour_paper_workloads(velocity, table, test):
    """Sec. 3, the paper's grid of workloads at q = 8 points per wavelength,
    n = 127 (omega/2pi = 16), alpha = 2, b = d = 12, left GMRES to 1e-3:
    velocity fields lens / vertical waveguide / random, forces Test 1 (point
    source at (0.5, 0.125)) and Test 2 (wave packet from (0.125, 0.125) along
    (1, 1)).  Synthetic stand-ins for the paper's fields: the iteration count
    must stay within the paper's count for the same table and test."""
    with open(os.path.join(GOLDEN, "paper_2d_iterations.json")) as fh:
        gold = json.load(fh)
    rows = [r for t in gold["tables"] if t["table"] == table for r in t["rows"] if r["n"] == 127 and r["test"] == test]
    assert len(rows) == 1
    n, omega = 127, 2 * np.pi * 16
    c = {"lens": I.lens_velocity(n), "waveguide": I.waveguide_velocity(n), "random": I.random_velocity(n, 0)}[velocity]
    f = (I.centered_source(n, center=(0.5, 0.125)) if test == 1 else I.wave_packet(n, omega))[0]
    A0 = H.helmholtz_matrix(c, omega, 12, 20.0, 0.0)
    st = S.setup(c, omega, 12, 12, 12, 2.0, 20.0)
    P = lambda v: S.apply(st, v.reshape(n, n)).ravel()
    _, it, _ = K.gmres_left(lambda v: A0 @ v, P, f.ravel(), tol=1e-3, maxit=200)
    assert 1 <= it <= rows[0]["n_iter"]


def test_workload_inputs_shapes():
    """The waveguide is constant along x2 and slowest on x1 = 1/2; the packet
    has unit peak amplitude at its centre and one wavelength of envelope."""
    n = 63
    c = I.waveguide_velocity(n)
    assert np.allclose(c, c[0:1, :])
    assert np.argmin(c[0]) == (n - 1) // 2
    f = I.wave_packet(n, 2 * np.pi * 8)[0]
    h = 1.0 / (n + 1)
    j = int(round(0.125 / h)) - 1
    assert abs(abs(f[j, j]) - 1.0) < 1e-12
