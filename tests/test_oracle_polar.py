"""Pins of the polar scattering oracle (Sec. 3, "Scattering problem", Table
2DRAD; oracle/polar.py): values the paper prints (the grid sizes of Table
2DRAD), the closed-form field scattered by a sound-soft disk, the exact limit
of the radial sweep, and planted slips that must fail.  CPU only."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import krylov as K
from oracle import polar as P

C = 20.0


def test_grid_matches_table_2drad():
    """q = 8 points per wavelength radially and on the outer circle gives the
    five grids printed in Table 2DRAD."""
    printed = {16: (45, 403), 32: (90, 805), 64: (180, 1609), 128: (359, 3217), 256: (717, 6434)}
    for f, (n_r, n_t) in printed.items():
        g = P.PolarGrid.for_frequency(f, 8)
        assert (g.n_r, g.n_t) == (n_r, n_t)


def test_operator_is_complex_symmetric_and_periodic():
    g = P.PolarGrid(12, 40)
    op = P.scattering_operator(g, 2 * np.pi * 4.0, 4, C)
    A = op.A
    assert abs(A - A.T).max() == 0.0
    # angle 0 couples to angle n_t - 1 on every ring (periodic in theta)
    for i in range(g.n_r):
        assert A[i * g.n_t, i * g.n_t + g.n_t - 1] != 0
    # a constant field on a ring with no PML: the angular part vanishes, the
    # row sum is the radial part and the mass term
    x = np.ones(A.shape[0])
    y = A @ x
    i = 3
    assert np.allclose(y[i * g.n_t:(i + 1) * g.n_t], y[i * g.n_t])


def scattering_error(f2pi, q, profile=None):
    """Relative error of the discrete plane-wave scattering against the Bessel
    series on the rings inside the PML's inner edge."""
    g = P.PolarGrid.for_frequency(f2pi, q)
    om = 2 * np.pi * f2pi
    bp = q
    prof = profile(g, bp) if profile is not None else P.boundary_profile(g, bp, C)
    op = P.RingOperator(g, om, 1.0, 1, g.n_r, prof)
    rhs = P.disk_rhs(op, -P.plane_wave(g, om, g.r0))
    u = spla.spsolve(op.A.tocsc(), rhs).reshape(g.n_r, g.n_t)
    eta = bp * g.h_r
    rings = [i for i in range(1, g.n_r + 1) if g.r(i) < g.r1 - eta]
    ex = np.array([P.exact_plane_wave_scattering(g, om, g.r(i)) for i in rings])
    return float(np.linalg.norm(u[[i - 1 for i in rings]] - ex) / np.linalg.norm(ex))


def test_plane_wave_scattering_matches_bessel_series():
    """Second order: halving h cuts the error about fourfold (PML one
    wavelength wide, C = 20)."""
    e16, e32 = scattering_error(4.0, 16), scattering_error(4.0, 32)
    assert e32 < 3e-3
    assert e16 / e32 > 3.0


def test_planted_slips_fail_the_series_pin():
    good = scattering_error(4.0, 32)
    # an amplifying PML (sigma of the wrong sign)
    amp = lambda g, bp: (lambda r: tuple(-v for v in P.boundary_profile(g, bp, C)(r)))
    assert scattering_error(4.0, 32, amp) > 0.5
    # r instead of the stretched radius r~ in the couplings
    flat = lambda g, bp: (lambda r: (P.boundary_profile(g, bp, C)(r)[0], 0.0 * np.asarray(r)))
    assert scattering_error(4.0, 32, flat) > 3.0 * good


def test_radial_sweep_with_cut_windows_is_a_direct_solve():
    """Every window reaching the PML boundary keeps the operator's own profile:
    each T~ is the exact Schur inverse and Algorithm 4 is A^{-1}."""
    g = P.PolarGrid(30, 96)
    om = 2 * np.pi * 4.0
    rng = np.random.default_rng(3)
    sw = P.RadialSweep(g, om, 6, g.n_r + 1, 4, C)
    r = rng.standard_normal(g.n_r * g.n_t) + 1j * rng.standard_normal(g.n_r * g.n_t)
    u = sw.apply(r)
    ref = spla.spsolve(sw.A.A.tocsc(), r)
    assert np.linalg.norm(u - ref) / np.linalg.norm(ref) < 1e-10


@pytest.mark.parametrize("field", ["green", "plane"])
def test_sweep_preconditions_the_table_2drad_problem(field):
    """Grid of the first row of Table 2DRAD (omega/2pi = 16, q = 8, 45 x 403),
    b_p = b = d = 8: FGMRES to 1e-3 within the paper's 7 iterations for both
    incident fields; with no moving-PML layer (b = 1) it does not converge
    within 40."""
    f2pi = 16.0
    g = P.PolarGrid.for_frequency(f2pi, 8)
    om = 2 * np.pi * f2pi
    uinc = P.point_source_field(g, om, g.r0) if field == "green" else P.plane_wave(g, om, g.r0)
    sw = P.RadialSweep(g, om, 8, 8, 8, C)
    rhs = P.disk_rhs(sw.A, -uinc)
    x, it, _ = K.fgmres(lambda v: sw.A.A @ v, sw.apply, rhs, tol=1e-3, restart=30, maxit=200)
    assert it <= 7
    assert np.linalg.norm(rhs - sw.A.A @ x) <= 1e-3 * np.linalg.norm(rhs)
    bare = P.RadialSweep(g, om, 8, 1, 4, C)
    _, it_bare, _ = K.fgmres(lambda v: bare.A.A @ v, bare.apply, rhs, tol=1e-3, restart=30, maxit=40)
    assert it_bare >= 40


@pytest.mark.parametrize("field", ["green", "plane"])
def test_sweep_preconditions_the_second_table_2drad_row(field):
    """Second row of Table 2DRAD (omega/2pi = 32, 90 x 805) with PML and
    moving PML 1.5 wavelengths wide (b_p = b = d = 12): within the paper's 7
    iterations.  (One wavelength, b_p = b = d = 8, takes 11 here.)"""
    f2pi = 32.0
    g = P.PolarGrid.for_frequency(f2pi, 8)
    om = 2 * np.pi * f2pi
    uinc = P.point_source_field(g, om, g.r0) if field == "green" else P.plane_wave(g, om, g.r0)
    sw = P.RadialSweep(g, om, 12, 12, 12, C)
    rhs = P.disk_rhs(sw.A, -uinc)
    x, it, _ = K.fgmres(lambda v: sw.A.A @ v, sw.apply, rhs, tol=1e-3, restart=30, maxit=200)
    assert it <= 7
    assert np.linalg.norm(rhs - sw.A.A @ x) <= 1e-3 * np.linalg.norm(rhs)
