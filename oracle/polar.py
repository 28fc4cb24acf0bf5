"""Polar-grid scattering by a sound-soft disk with a radial sweep (oracle;
test infrastructure only: imported by ``tests/`` alone, and independent of
the CUDA path, which does not implement this variant).

Paper passage restated here: Sec. 3, "Scattering problem" (Table 2DRAD).  The
scattered field u around the disk r < r0 satisfies
    (1/r)(r u_r)_r + (1/r^2) u_thth + (omega^2/c^2) u = f,
    u(r0, th) = -u_inc(r0, th),
with the Sommerfeld condition at infinity, replaced by a PML at r = r1; the
sweeping preconditioner runs radially from r1 to r0.  c = 1, r0 = 0.15,
r1 = 0.5, q points per wavelength; incident fields: the Green's function
centred at (-0.2, 0.2) and the plane wave exp(-i omega x2).

Readings (the passage gives no formulas beyond the PDE):

* Grid: rings r_i = r0 + i h_r, h_r = (r1 - r0)/(n_r + 1), unknowns on
  i = 1..n_r (ring 0 carries the disk's Dirichlet data, ring n_r + 1 = r1 is a
  zero Dirichlet boundary behind the PML); angles th_j = j h_t, h_t = 2 pi/n_t,
  periodic.  Unknowns ring by ring, angle fastest.  With
  n_r = ceil((r1 - r0) q / lambda) and n_t = ceil(2 pi r1 q / lambda) this
  reproduces the five grid sizes of Table 2DRAD (45 x 403 at omega/2pi = 16
  up to 717 x 6434 at 256, q = 8).
* PML: the quadratic profile of Eq. sigma in the radial coordinate,
  sigma(r) = (C/eta)((r - (r1 - eta))/eta)^2 on [r1 - eta, r1], eta = b_p h_r,
  and the complex stretched radius r~ = r + (i/omega) int_r0^r sigma, so that
  with s = (1 + i sigma/omega)^(-1) (the stretch factor of Sec. 2.1) the
  operator is (s/r~) d_r(r~ s d_r u) + (1/r~^2) u_thth + (omega^2/c^2) u.  Each
  row is multiplied by r~_i/s_i, which makes the 5-point matrix complex
  symmetric: radial couplings r~ s / h_r^2 at the half rings, angular
  couplings 1/(s r~ h_t^2), diagonal r~ omega^2/(s c^2) minus the couplings.
* Sweep (Algorithms 3 and 4, single front, d rings per step): the first
  block F is the b_p outermost rings (the PML), solved exactly; every later
  block of d rings (the last takes the remainder, ending at ring 1) is solved
  on a window of its rings and the b - 1 rings outside it, with the moving
  profile of Eq. helma anchored at the block's outer ring,
  sigma_m(r) = (C/eta_b)((r - r_hi)/eta_b)^2, eta_b = b h_r, and a zero
  Dirichlet ring just outside the window.  A window that would reach past ring
  n_r is cut there and keeps the operator's own profile (the exact Schur
  inverse).
* The right-hand side of the scattering problem is the disk's data moved to
  ring 1: rhs = -a_{1/2} u0 with u0 = -u_inc(r0, th).

Pins (tests/test_oracle_polar.py): the closed-form field scattered by a
sound-soft disk (Bessel/Hankel series) with second-order convergence; the
sweep with every window cut equals a sparse direct solve; planted slips (an
amplifying PML, r instead of r~ in the angular coupling) fail the series pin;
FGMRES preconditioned by the sweep converges in about the paper's iteration
count at the grid of Table 2DRAD.
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla
import scipy.special as ss


class PolarGrid:
    """Rings r_i = r0 + i h_r (i = 0..n_r + 1) and angles th_j = j h_t."""

    def __init__(self, n_r, n_t, r0=0.15, r1=0.5):
        self.n_r, self.n_t, self.r0, self.r1 = int(n_r), int(n_t), float(r0), float(r1)
        self.h_r = (self.r1 - self.r0) / (self.n_r + 1)
        self.h_t = 2.0 * np.pi / self.n_t
        self.theta = np.arange(self.n_t) * self.h_t

    def r(self, i):
        return self.r0 + np.asarray(i, dtype=np.float64) * self.h_r

    @staticmethod
    def for_frequency(omega_over_2pi, q, r0=0.15, r1=0.5, c=1.0):
        """The grid of Table 2DRAD: q points per wavelength radially and on the
        outer circle."""
        lam = c / omega_over_2pi
        n_r = int(np.ceil((r1 - r0) * q / lam - 1e-9))
        n_t = int(np.ceil(2.0 * np.pi * r1 * q / lam - 1e-9))
        return PolarGrid(n_r, n_t, r0, r1)


def quadratic_profile(r, start, eta, C):
    """sigma(r) = (C/eta)((r - start)/eta)^2 for r > start, 0 below, and its
    integral from r0 (any point below `start`) to r."""
    r = np.asarray(r, dtype=np.float64)
    t = np.clip(r - start, 0.0, None)
    return (C / eta) * (t / eta) ** 2, (C / (3.0 * eta ** 3)) * t ** 3


def boundary_profile(grid, bp, C):
    """Profile of the PML at r1 (b_p rings wide) as a function of r."""
    eta = bp * grid.h_r
    return lambda r: quadratic_profile(r, grid.r1 - eta, eta, C)


class RingOperator:
    """5-point polar operator on rings ilo..ihi (inclusive) with zero
    Dirichlet rings ilo - 1 and ihi + 1, built from a profile function that
    returns (sigma(r), int_r0^r sigma)."""

    def __init__(self, grid, omega, c, ilo, ihi, profile):
        self.grid, self.omega, self.ilo, self.ihi = grid, omega, ilo, ihi
        nr = ihi - ilo + 1
        nt = grid.n_t
        self.nr, self.nt = nr, nt
        ri = grid.r(np.arange(ilo, ihi + 1))
        rh = grid.r(np.arange(ilo, ihi + 2) - 0.5)       # half rings ilo-1/2 .. ihi+1/2
        sig_i, int_i = profile(ri)
        sig_h, int_h = profile(rh)
        s_i = 1.0 / (1.0 + 1j * sig_i / omega)
        s_h = 1.0 / (1.0 + 1j * sig_h / omega)
        rt_i = ri + 1j * int_i / omega
        rt_h = rh + 1j * int_h / omega
        self.a_half = rt_h * s_h / grid.h_r ** 2          # radial couplings at the half rings
        self.b_ring = 1.0 / (s_i * rt_i * grid.h_t ** 2)  # angular couplings per ring
        c = np.asarray(c, dtype=np.float64)
        cr = c[ilo - 1: ihi, :] if c.ndim == 2 else np.full((nr, nt), float(c))
        diag = (rt_i / s_i)[:, None] * omega ** 2 / cr ** 2
        diag = diag - (self.a_half[:-1] + self.a_half[1:])[:, None] - 2.0 * self.b_ring[:, None]
        N = nr * nt
        idx = np.arange(N).reshape(nr, nt)
        rows, cols, vals = [idx.ravel()], [idx.ravel()], [diag.ravel()]
        # angular neighbours (periodic)
        for dj in (1, -1):
            rows.append(idx.ravel())
            cols.append(np.roll(idx, -dj, axis=1).ravel())
            vals.append(np.repeat(self.b_ring, nt))
        # radial neighbours inside the range
        if nr > 1:
            up = idx[:-1].ravel()
            dn = idx[1:].ravel()
            a = np.repeat(self.a_half[1:-1], nt)
            rows += [up, dn]
            cols += [dn, up]
            vals += [a, a]
        self.A = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(N, N))

    def inner_coupling(self):
        """Coefficient a_{ilo - 1/2} coupling ring ilo to ring ilo - 1."""
        return self.a_half[0]

    def outer_coupling(self):
        """Coefficient a_{ihi + 1/2} coupling ring ihi to ring ihi + 1."""
        return self.a_half[-1]


def scattering_operator(grid, omega, bp, C, c=1.0):
    """The global operator A on rings 1..n_r with the boundary PML."""
    return RingOperator(grid, omega, c, 1, grid.n_r, boundary_profile(grid, bp, C))


def disk_rhs(op, u0):
    """Right-hand side of A u = rhs for the Dirichlet data u0(th) on ring 0
    (the disk) and no source: -a_{1/2} u0 on ring 1."""
    rhs = np.zeros(op.nr * op.nt, dtype=np.complex128)
    rhs[: op.nt] = -op.inner_coupling() * np.asarray(u0, dtype=np.complex128)
    return rhs


# ---------------------------------------------------------------- incident fields
def plane_wave(grid, omega, r):
    """exp(-i omega x2) on the circle of radius r (c = 1)."""
    return np.exp(-1j * omega * r * np.sin(grid.theta))


def point_source_field(grid, omega, r, x0=(-0.2, 0.2)):
    """Free-space Green's function (i/4) H0^(1)(omega |x - x0|) on the circle of
    radius r (c = 1), the paper's first incident field."""
    x = r * np.cos(grid.theta) - x0[0]
    y = r * np.sin(grid.theta) - x0[1]
    return 0.25j * ss.hankel1(0, omega * np.hypot(x, y))


def exact_plane_wave_scattering(grid, omega, r, nterms=None):
    """Field scattered by the sound-soft disk r0 from exp(-i omega x2) (c = 1)
    on the circle of radius r: with the Jacobi-Anger expansion
    exp(-i k r sin th) = sum_n (-1)^n J_n(k r) e^(i n th),
    u_s = -sum_n (-1)^n J_n(k r0)/H_n(k r0) H_n(k r) e^(i n th), H_n = H_n^(1)
    (outgoing for the time factor e^(-i omega t))."""
    k = omega
    if nterms is None:
        nterms = int(k * grid.r1) + 40
    n = np.arange(-nterms, nterms + 1)
    coef = -((-1.0) ** np.abs(n)) * ss.jv(n, k * grid.r0) / ss.hankel1(n, k * grid.r0) * ss.hankel1(n, k * r)
    return (coef[None, :] * np.exp(1j * np.outer(grid.theta, n))).sum(axis=1)


# ---------------------------------------------------------------- radial sweep
class RadialSweep:
    """Algorithms 3 and 4 on rings, single front from r1 toward r0."""

    def __init__(self, grid, omega, bp, b, dL, C, c=1.0, Cm=None):
        self.grid, self.omega = grid, omega
        Cm = C if Cm is None else Cm
        n = grid.n_r
        prof_b = boundary_profile(grid, bp, C)
        self.A = scattering_operator(grid, omega, bp, C, c)
        blocks = [(max(1, n - bp + 1), n)]                    # F: the PML rings
        hi = n - bp
        while hi >= 1:
            lo = max(1, hi - dL + 1)
            blocks.append((lo, hi))
            hi = lo - 1
        self.blocks = blocks
        self.windows = []
        for k, (lo, hi) in enumerate(blocks):
            if k == 0:
                op = RingOperator(grid, omega, c, lo, hi, prof_b)
            else:
                whi = hi + b - 1
                if whi >= n:                                   # cut at the PML boundary: exact
                    op = RingOperator(grid, omega, c, lo, n, prof_b)
                else:
                    eta_b = b * grid.h_r
                    r_hi = grid.r(hi)
                    op = RingOperator(grid, omega, c, lo, whi,
                                      lambda r, r_hi=r_hi, eta_b=eta_b: quadratic_profile(r, r_hi, eta_b, Cm))
            self.windows.append((op, spla.splu(op.A.tocsc())))
        # couplings of the global operator between consecutive blocks: block k's
        # outer ring hi_k and block k-1's inner ring hi_k + 1
        self.coupling = [None] + [self.A.a_half[hi] for (lo, hi) in blocks[1:]]

    def _ring_slice(self, lo, hi):
        return slice((lo - 1) * self.grid.n_t, hi * self.grid.n_t)

    def _tilde_solve(self, k, g):
        """T~_k g: the window solve with g on the block's rings (which come first
        in the window) and zero on the extra rings, restricted to the block."""
        op, lu = self.windows[k]
        lo, hi = self.blocks[k]
        nb = (hi - lo + 1) * self.grid.n_t
        rhs = np.zeros(op.nr * op.nt, dtype=np.complex128)
        rhs[:nb] = g
        return lu.solve(rhs)[:nb]

    def apply(self, r):
        """u = M r (Algorithm 4: forward sweep toward r0, then back)."""
        nt = self.grid.n_t
        r = np.asarray(r, dtype=np.complex128)
        K = len(self.blocks)
        v = []
        for k, (lo, hi) in enumerate(self.blocks):
            g = r[self._ring_slice(lo, hi)].copy()
            if k > 0:
                # -A_{k,k-1} v_{k-1}: block k's outer ring couples to block k-1's inner ring
                g[-nt:] -= self.coupling[k] * v[k - 1][:nt]
            v.append(self._tilde_solve(k, g))
        u = [None] * K
        u[K - 1] = v[K - 1]
        for k in range(K - 2, -1, -1):
            lo, hi = self.blocks[k]
            g = np.zeros((hi - lo + 1) * nt, dtype=np.complex128)
            # A_{k,k+1} u_{k+1}: block k's inner ring couples to block k+1's outer ring
            g[:nt] = self.coupling[k + 1] * u[k + 1][-nt:]
            u[k] = v[k] - self._tilde_solve(k, g)
        out = np.empty(self.grid.n_r * nt, dtype=np.complex128)
        for k, (lo, hi) in enumerate(self.blocks):
            out[self._ring_slice(lo, hi)] = u[k]
        return out
