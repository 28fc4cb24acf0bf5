"""2D PML-stretched Helmholtz operator, complex128 (oracle; test infrastructure only).

Paper passages restated here (Engquist & Ying 2010, Sec. 2.1):

* Eq. sigma: the quadratic absorption profile
      sigma(t) = (C/eta) ((t - eta)/eta)^2   on [0, eta],
                 0                            on [eta, 1 - eta],
                 (C/eta) ((t - 1 + eta)/eta)^2 on [1 - eta, 1].
  Every experiment of the paper puts the PML on all four sides, so both
  axes use this two-sided profile by default; the one-sided sigma_2 of Sec.
  2.1 (``pml_sigma_one_sided``, ``dirichlet_top=True``) gives the
  Dirichlet-top formulation that Algorithms 3 and 4 are written for.
* Stretch factors s_k(x_k) = (1 + i sigma_k(x_k)/omega)^(-1), with the real
  frequency omega (the shift alpha of Eq. helmalpha changes only the mass
  term).
* Eq. helmd: the 5-point scheme on the grid p_ij = (ih, jh), h = 1/(n+1),
  1 <= i, j <= n, unknowns ordered row by row with x1 fastest.  Off-diagonal
  coefficients (1/h^2)(s1/s2) at (i +- 1/2, j) and (1/h^2)(s2/s1) at
  (i, j +- 1/2); the diagonal is omega_*^2 / ((s1 s2)_ij c_ij^2) minus the sum
  of the four off-diagonal coefficients, where omega_* = omega for A and
  omega + i alpha for A_alpha (Eq. helmalpha).  Neighbours outside
  1..n are zero (Dirichlet) but their coefficients still enter the diagonal.
  Half-point coefficients evaluate s at the half-point coordinate.
"""
import numpy as np
import scipy.sparse as sp


def pml_sigma(t, eta, C):
    """Two-sided quadratic profile of Eq. sigma at coordinates ``t`` (array)."""
    t = np.asarray(t, dtype=np.float64)
    out = np.zeros_like(t)
    lo = t <= eta
    hi = t >= 1.0 - eta
    out[lo] = (C / eta) * ((t[lo] - eta) / eta) ** 2
    out[hi] = (C / eta) * ((t[hi] - 1.0 + eta) / eta) ** 2
    return out


def pml_sigma_one_sided(t, eta, C):
    """sigma_2 of Eq. sigma: the quadratic ramp near x2 = 0 only (the
    Dirichlet-top formulation of Sec. 2.1), zero on [eta, 1]."""
    t = np.asarray(t, dtype=np.float64)
    out = np.zeros_like(t)
    lo = t <= eta
    out[lo] = (C / eta) * ((t[lo] - eta) / eta) ** 2
    return out


def stretch(sigma, omega):
    """s = (1 + i sigma/omega)^(-1) (Sec. 2.1)."""
    return 1.0 / (1.0 + 1j * np.asarray(sigma) / omega)


def axis_stretch(n, bp, C, omega, one_sided=False):
    """Stretch factors of one axis at integer points k h (k = 0..n+1) and at
    half points (k + 1/2) h (k = 0..n).  eta = bp*h is the boundary PML width;
    ``one_sided`` takes sigma_2 of Eq. sigma (PML at 0 only).

    Returns (s_int, s_half) with s_int[k] = s(k h), s_half[k] = s((k+1/2) h).
    """
    h = 1.0 / (n + 1)
    eta = bp * h
    sig = pml_sigma_one_sided if one_sided else pml_sigma
    k = np.arange(n + 2, dtype=np.float64)
    s_int = stretch(sig(k * h, eta, C), omega)
    s_half = stretch(sig((k[: n + 1] + 0.5) * h, eta, C), omega)
    return s_int, s_half


def row_coefficients(c_rows, omega, alpha, h, s1, s2_int, s2_up, s2_dn):
    """Eq. helmd coefficients for a set of grid rows (all n columns).

    ``c_rows``: (w, n) velocities of the rows; ``s1`` = (s_int, s_half) table
    of the x1 axis; ``s2_int``, ``s2_up``, ``s2_dn``: (w,) values of the x2
    stretch at the rows, at the half points above (j + 1/2) and below
    (j - 1/2).  Returns dict E, W, N, S, D of shape (w, n).
    """
    c_rows = np.asarray(c_rows, dtype=np.float64)
    w, n = c_rows.shape
    s1_int, s1_half = s1
    i = np.arange(1, n + 1)
    s1_i = s1_int[i][None, :]          # s1(i h)
    s1_ip = s1_half[i][None, :]        # s1((i + 1/2) h)
    s1_im = s1_half[i - 1][None, :]    # s1((i - 1/2) h)
    s2_j = np.asarray(s2_int)[:, None]
    s2_jp = np.asarray(s2_up)[:, None]
    s2_jm = np.asarray(s2_dn)[:, None]
    ones = np.ones((w, n))
    E = (s1_ip / s2_j) / h**2 * ones
    W = (s1_im / s2_j) / h**2 * ones
    N = (s2_jp / s1_i) / h**2 * ones
    S = (s2_jm / s1_i) / h**2 * ones
    wst = omega + 1j * alpha
    D = wst**2 / (s1_i * s2_j * c_rows**2) - (E + W + N + S)
    return dict(E=E, W=W, N=N, S=S, D=D)


def stencil_coefficients(c, omega, bp, C, alpha=0.0, dirichlet_top=False):
    """Coefficients of Eq. helmd on the full grid.

    ``c`` is the (n, n) velocity array indexed [j-1, i-1] (row j = x2 index,
    column i = x1 index).  Returns a dict of (n, n) complex arrays
    E, W, N, S (couplings to (i+1,j), (i-1,j), (i,j+1), (i,j-1)) and D (the
    diagonal of A_alpha; alpha = 0 gives A).  ``dirichlet_top``: the
    formulation of Sec. 2.1 (sigma_2 one-sided, no PML at x2 = 1; the zero
    Dirichlet values outside the grid are the boundary condition there).
    """
    c = np.asarray(c, dtype=np.float64)
    n = c.shape[0]
    assert c.shape == (n, n)
    h = 1.0 / (n + 1)
    s1 = axis_stretch(n, bp, C, omega)
    s2_int, s2_half = axis_stretch(n, bp, C, omega, one_sided=dirichlet_top)
    j = np.arange(1, n + 1)
    return row_coefficients(c, omega, alpha, h, s1, s2_int[j], s2_half[j], s2_half[j - 1])


def assemble(coef):
    """Sparse matrix of Eq. helmd from ``stencil_coefficients`` output.

    Row index of (i, j) is (j-1) n + (i-1) (the paper's ordering).
    """
    D = coef["D"]
    n = D.shape[0]
    N2 = n * n
    idx = np.arange(N2).reshape(n, n)
    rows, cols, vals = [idx.ravel()], [idx.ravel()], [D.ravel()]
    # east: (i,j) -> (i+1,j), valid for i < n
    rows.append(idx[:, :-1].ravel()); cols.append(idx[:, 1:].ravel()); vals.append(coef["E"][:, :-1].ravel())
    rows.append(idx[:, 1:].ravel()); cols.append(idx[:, :-1].ravel()); vals.append(coef["W"][:, 1:].ravel())
    rows.append(idx[:-1, :].ravel()); cols.append(idx[1:, :].ravel()); vals.append(coef["N"][:-1, :].ravel())
    rows.append(idx[1:, :].ravel()); cols.append(idx[:-1, :].ravel()); vals.append(coef["S"][1:, :].ravel())
    A = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(N2, N2), dtype=np.complex128)
    return A


def helmholtz_matrix(c, omega, bp, C, alpha=0.0, dirichlet_top=False):
    """A (alpha = 0) or A_alpha of Eq. helmd / Eq. helmalpha as a CSR matrix."""
    return assemble(stencil_coefficients(c, omega, bp, C, alpha, dirichlet_top))


def apply_stencil(coef, x):
    """y = A x evaluated point by point from the five coefficients of Eq. helmd.

    ``x`` has shape (..., n, n) (any leading RHS axes).  Written directly from
    the stencil so that it is independent of ``assemble``.
    """
    x = np.asarray(x, dtype=np.complex128)
    y = coef["D"] * x
    y[..., :, :-1] += coef["E"][:, :-1] * x[..., :, 1:]
    y[..., :, 1:] += coef["W"][:, 1:] * x[..., :, :-1]
    y[..., :-1, :] += coef["N"][:-1, :] * x[..., 1:, :]
    y[..., 1:, :] += coef["S"][1:, :] * x[..., :-1, :]
    return y
