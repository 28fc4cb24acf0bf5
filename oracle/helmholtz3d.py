"""3D PML-stretched Helmholtz operator and slab sweep, complex128 (oracle; test infrastructure only).

Restates Sec. 4 of Engquist & Ying (2010):

* Eq. helmd3: the 7-point scheme on p_ijk = (ih, jh, kh), h = 1/(n+1),
  unknowns ordered with x1 fastest, then x2, then x3 (index
  (k-1) n^2 + (j-1) n + (i-1)).  Off-diagonal coefficients
  (1/h^2) s1/(s2 s3) at (i +- 1/2, j, k), s2/(s1 s3) at (i, j +- 1/2, k),
  s3/(s1 s2) at (i, j, k +- 1/2); the diagonal is
  omega_*^2 / ((s1 s2 s3)_ijk c_ijk^2) minus the sum of the six, with
  omega_* = omega for A and omega + i alpha for A_alpha.  Neighbours outside
  1..n are zero.  Every 3D experiment puts the PML on all sides, so all
  three axes use the two-sided profile of Eq. sigma (as in 2D).
* The block-tridiagonal form in x3 layers (n^2 unknowns per layer, diagonal
  couplings between layers) and the moving-PML subproblem Eq. helma3 on the
  window of b layers ending at the block: x3 stretch with the one-sided
  profile sigma_3(x3 - (m-b)h), zero Dirichlet values outside.
* Algorithms 5 and 6 with the two-front pattern and d layers per step of
  Sec. 2.3 (the 3D experiments sweep with two fronts).  T~_B is computed with
  an exact sparse LU of H_B (SciPy's SuperLU) instead of the paper's
  multifrontal LDL^t; both are exact solvers of the same H_B, so T~_B and
  M_alpha are the same operator.

The block partition, the moving profile and the window rules are those of
``sweep2d`` with rows read as x3 layers; they are reused from there.  The
readings listed there apply here unchanged.  Pins: the x3 moving profile is
the 2D one (its hand-computed values are checked through
``window_x3_stretch``); full windows reproduce A_alpha^{-1}; exact Schur
complements reproduce a sparse direct solve; the Green's function
-exp(ikr)/(4 pi r) converges at second order.
"""
from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import helmholtz2d as H2
from . import sweep2d as S2


def axis_tables(n, bp, C, omega):
    """s at integer points k h (k = 0..n+1) and at half points (k+1/2) h (k = 0..n)."""
    return H2.axis_stretch(n, bp, C, omega)


def coefficients(c, omega, bp, C, alpha=0.0, s3=None):
    """Eq. helmd3 coefficients on the grid of ``c`` (shape (nz, n, n), indexed
    [k-1, j-1, i-1]).  ``s3`` = (s_int, s_up, s_dn) per layer overrides the x3
    stretch (moving-PML windows); by default the boundary profile of the full
    grid.  Returns arrays E, W, N, S, U, Dn (couplings to (i+1), (i-1),
    (j+1), (j-1), (k+1), (k-1)) and the diagonal D, each of shape (nz, n, n)."""
    c = np.asarray(c, dtype=np.float64)
    nz, n, _ = c.shape
    h = 1.0 / (n + 1)
    si, sh = axis_tables(n, bp, C, omega)
    idx = np.arange(1, n + 1)
    s1 = si[idx][None, None, :]
    s1p = sh[idx][None, None, :]          # s1((i+1/2)h)
    s1m = sh[idx - 1][None, None, :]      # s1((i-1/2)h)
    s2 = si[idx][None, :, None]
    s2p = sh[idx][None, :, None]
    s2m = sh[idx - 1][None, :, None]
    if s3 is None:
        kk = np.arange(1, nz + 1)
        s3i, s3p, s3m = si[kk], sh[kk], sh[kk - 1]
    else:
        s3i, s3p, s3m = s3
    s3i = np.asarray(s3i)[:, None, None]
    s3p = np.asarray(s3p)[:, None, None]
    s3m = np.asarray(s3m)[:, None, None]
    h2 = h * h
    E = s1p / (s2 * s3i) / h2 * np.ones((nz, n, n))
    W = s1m / (s2 * s3i) / h2 * np.ones((nz, n, n))
    N = s2p / (s1 * s3i) / h2 * np.ones((nz, n, n))
    S = s2m / (s1 * s3i) / h2 * np.ones((nz, n, n))
    U = s3p / (s1 * s2) / h2 * np.ones((nz, n, n))
    Dn = s3m / (s1 * s2) / h2 * np.ones((nz, n, n))
    wst = omega + 1j * alpha
    D = wst * wst / (s1 * s2 * s3i * c * c) - (E + W + N + S + U + Dn)
    return dict(E=E, W=W, N=N, S=S, U=U, Dn=Dn, D=D)


def assemble(coef):
    """Sparse matrix of Eq. helmd3 from ``coefficients`` output."""
    D = coef["D"]
    nz, n, _ = D.shape
    idx = np.arange(nz * n * n).reshape(nz, n, n)
    rows, cols, vals = [idx.ravel()], [idx.ravel()], [D.ravel()]

    def add(r, c_, v):
        rows.append(r.ravel()); cols.append(c_.ravel()); vals.append(v.ravel())

    add(idx[:, :, :-1], idx[:, :, 1:], coef["E"][:, :, :-1])
    add(idx[:, :, 1:], idx[:, :, :-1], coef["W"][:, :, 1:])
    add(idx[:, :-1, :], idx[:, 1:, :], coef["N"][:, :-1, :])
    add(idx[:, 1:, :], idx[:, :-1, :], coef["S"][:, 1:, :])
    add(idx[:-1], idx[1:], coef["U"][:-1])
    add(idx[1:], idx[:-1], coef["Dn"][1:])
    N3 = nz * n * n
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(N3, N3), dtype=np.complex128)


def helmholtz_matrix(c, omega, bp, C, alpha=0.0):
    """A (alpha = 0) or A_alpha of Eq. helmd3 as a CSR matrix."""
    return assemble(coefficients(c, omega, bp, C, alpha))


def window_x3_stretch(blk, n, bp, b, C, omega, full_window=False, Cm=None):
    """x3 stretch of H_B on the window layers (integer and half points),
    the moving profile of Eq. helma3 (same rules as the 2D x2 stretch)."""
    return S2.window_x2_stretch(blk, n, bp, b, C, omega, full_window, Cm)


@dataclass
class FactoredSlab:
    blk: S2.Block
    lu: object
    n: int

    def t_tilde(self, g):
        """T~_B g for g of shape (R, d, n, n) on the block layers lo..hi:
        H_B^{-1} of the vector that is zero on the other window layers,
        restricted to the block layers."""
        blk, n = self.blk, self.n
        R, d = g.shape[0], g.shape[1]
        off = blk.lo - blk.wlo
        rhs = np.zeros((R, blk.w, n, n), dtype=np.complex128)
        rhs[:, off:off + d] = g
        x = self.lu.solve(rhs.reshape(R, -1).T)
        x = x.T.reshape(R, blk.w, n, n)
        return x[:, off:off + d].copy()


def factor_slab(blk, c, omega, bp, b, C, alpha, full_window=False, Cm=None):
    """Sparse LU of the slab problem H_B (Eq. helma3 on the window)."""
    n = c.shape[1]
    s3 = window_x3_stretch(blk, n, bp, b, C, omega, full_window, Cm)
    cw = c[blk.wlo - 1:blk.whi]
    Hm = assemble(coefficients(cw, omega, bp, C, alpha, s3=s3)).tocsc()
    return FactoredSlab(blk, spla.splu(Hm), n)


@dataclass
class Setup:
    n: int
    lower: list
    upper: list
    middle: FactoredSlab
    Ucoup: np.ndarray     # coupling of layer k to k+1, shape (n, n, n) [k-1, j-1, i-1]


def setup(c, omega, bp, b, dL, alpha, C, full_window=False, Cm=None):
    """Algorithm 5 with two fronts and d layers per step: factor every slab."""
    c = np.asarray(c, dtype=np.float64)
    n = c.shape[0]
    lower, upper, middle = S2.partition(n, bp, b, dL, full_window)
    f = lambda blk: factor_slab(blk, c, omega, bp, b, C, alpha, full_window, Cm)
    coef = coefficients(c, omega, bp, C, alpha)
    return Setup(n, [f(B) for B in lower], [f(B) for B in upper], f(middle), coef["U"])


def apply(st, r):
    """Algorithm 6 with two fronts: u = M_alpha r, r of shape (R, n, n, n) or (n, n, n)."""
    squeeze = r.ndim == 3
    u = np.array(r, dtype=np.complex128).reshape((-1,) + r.shape[-3:]).copy()
    Uc = st.Ucoup
    lay = lambda B: slice(B.blk.lo - 1, B.blk.hi)
    v = {}
    for k, B in enumerate(st.lower):
        v[k, 0] = B.t_tilde(u[:, lay(B)])
        hi = B.blk.hi
        u[:, hi] -= Uc[hi - 1] * v[k, 0][:, -1]
    for k, B in enumerate(st.upper):
        v[k, 1] = B.t_tilde(u[:, lay(B)])
        lo = B.blk.lo
        u[:, lo - 2] -= Uc[lo - 2] * v[k, 1][:, 0]
    u[:, lay(st.middle)] = st.middle.t_tilde(u[:, lay(st.middle)])
    for k in range(len(st.lower) - 1, -1, -1):
        B = st.lower[k]
        hi = B.blk.hi
        g = np.zeros_like(v[k, 0])
        g[:, -1] = Uc[hi - 1] * u[:, hi]
        u[:, lay(B)] = v[k, 0] - B.t_tilde(g)
    for k in range(len(st.upper) - 1, -1, -1):
        B = st.upper[k]
        lo = B.blk.lo
        g = np.zeros_like(v[k, 1])
        g[:, 0] = Uc[lo - 2] * u[:, lo - 2]
        u[:, lay(B)] = v[k, 1] - B.t_tilde(g)
    return u[0] if squeeze else u


def apply_stencil(coef, x):
    """y = A x on arrays of shape (R, n, n, n) (zero outside the grid)."""
    x = np.asarray(x, dtype=np.complex128)
    y = coef["D"] * x
    y[..., :, :, :-1] += coef["E"][:, :, :-1] * x[..., :, :, 1:]
    y[..., :, :, 1:] += coef["W"][:, :, 1:] * x[..., :, :, :-1]
    y[..., :, :-1, :] += coef["N"][:, :-1, :] * x[..., :, 1:, :]
    y[..., :, 1:, :] += coef["S"][:, 1:, :] * x[..., :, :-1, :]
    y[..., :-1, :, :] += coef["U"][:-1] * x[..., 1:, :, :]
    y[..., 1:, :, :] += coef["Dn"][1:] * x[..., :-1, :, :]
    return y


def exact_apply(c, omega, bp, b, dL, alpha, C, f):
    """Algorithms 1-2 in the two-front layer-block order with exact Schur
    complements (dense; tiny n only): reproduces A_alpha^{-1} f."""
    c = np.asarray(c, dtype=np.float64)
    n = c.shape[0]
    A = helmholtz_matrix(c, omega, bp, C, alpha).toarray()
    lower, upper, middle = S2.partition(n, bp, b, dL)
    idx = lambda B: np.arange((B.lo - 1) * n * n, B.hi * n * n)
    T = {}
    for front in (lower, upper):
        prev = None
        for B in front:
            I = idx(B)
            S = A[np.ix_(I, I)].copy()
            if prev is not None:
                P = idx(prev)
                S -= A[np.ix_(I, P)] @ T[prev.lo] @ A[np.ix_(P, I)]
            T[B.lo] = np.linalg.inv(S)
            prev = B
    I = idx(middle)
    S = A[np.ix_(I, I)].copy()
    for front in (lower, upper):
        P = idx(front[-1])
        S -= A[np.ix_(I, P)] @ T[front[-1].lo] @ A[np.ix_(P, I)]
    T[middle.lo] = np.linalg.inv(S)
    u = np.array(f, dtype=np.complex128).reshape(-1).copy()
    for front in (lower, upper):
        for k in range(len(front)):
            B = front[k]
            nxt = front[k + 1] if k + 1 < len(front) else middle
            I, J = idx(B), idx(nxt)
            u[J] -= A[np.ix_(J, I)] @ (T[B.lo] @ u[I])
    for B in lower + upper + [middle]:
        I = idx(B)
        u[I] = T[B.lo] @ u[I]
    for front in (lower, upper):
        for k in range(len(front) - 1, -1, -1):
            B = front[k]
            nxt = front[k + 1] if k + 1 < len(front) else middle
            I, J = idx(B), idx(nxt)
            u[I] -= T[B.lo] @ (A[np.ix_(I, J)] @ u[J])
    return u.reshape(n, n, n)
