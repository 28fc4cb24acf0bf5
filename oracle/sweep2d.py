"""Moving-PML sweeping preconditioner in 2D, complex128 (oracle; test infrastructure only).

Restates, in the paper's order and notation (Engquist & Ying 2010):

* Sec. 2.3, two-front pattern and "several layers per step": the rows are
  split into a front F = rows 1..b_p, an end E = rows n-b_p+1..n, lower blocks
  of d rows swept upward from F, upper blocks swept downward from E, and a
  middle block that receives moving PMLs on both sides.
* Sec. 2.2, Eq. helma: the moving-PML subproblem H_m of a block lives on the
  window of the block's rows plus b-1 rows on the already-eliminated side,
  with x2 stretch s2^m(x2) = (1 + i sigma(x2 - (lo-b)h)/omega)^(-1) whose
  one-sided quadratic profile vanishes at the block's first row; zero
  Dirichlet values outside the window.  The approximate Schur inverse
  T~_m g is the restriction to the block rows of H_m^{-1} (0, ..., 0, g).
* Algorithm 3: the LU factorisation of P_m H_m P_m^t in the x2-first
  ordering (a band matrix with half band width equal to the window height),
  one factorisation per block, blocks independent.
* Algorithm 4: the forward sweep u_{m+1} -= A_{m+1,m} T~_m u_m, the diagonal
  step u_m = T~_m u_m, and the backward sweep u_m -= T~_m A_{m,m+1} u_{m+1}.
* Algorithms 1 and 2 (``exact_setup`` / ``exact_apply``): the same block
  elimination with the exact Schur complements S_m, used as a pin.

Readings of passages the paper leaves open (each also a constant of the CUDA
path, chosen independently there):
  - the boundary PML profile is two-sided in both axes (all experiments have
    PML on all sides); s uses the real omega; alpha only shifts the mass term;
  - the moving profile uses eta_b = b h with the same constant C as the
    boundary PML; the block window for d > 1 is the block rows plus b - 1
    rows on the eliminated side; the middle is the single layer (n+1)/2 with
    both profiles, and the last block of each front takes the remainder
    rows when d does not divide them;
  - the half band width of P_m H_m P_m^t is the window height (the paper's
    "b - 1 diagonals" is an off-by-one);
  - the LAPACK band LU pivots by rows; any exact solver defines the same T~.
* Sec. 2.1-2.2 as printed (``partition_single``, ``two_front=False``): the
  Dirichlet-top formulation, one-sided sigma_2, one upward sweep from F, the
  top block solved once (no middle layer).
* Sec. 2.2, buffer layers (``buffer``): k undamped rows between a block and
  its moving PML; a window that would cross the grid boundary is cut there
  and keeps the operator's own profile (the exact Schur inverse).

Pins (tests/): the moving profile against hand-computed values (b != b_p,
lower, upper and middle windows, with and without buffers) and against the
half-space Green's function it approximates (error falling in b and in k);
each T~ against a dense solve of H_B; the sweep algebra against sparse direct
solves in its exact limits (full windows, exact Schur complements, windows
cut by large buffers), for both formulations.
"""
from dataclasses import dataclass
import numpy as np
import scipy.linalg.lapack as lapack

from . import helmholtz2d as H


@dataclass
class Block:
    kind: str      # 'F', 'E', 'lower', 'upper', 'middle'
    lo: int        # first row of the block (1-based, inclusive)
    hi: int        # last row of the block
    wlo: int       # first row of the subproblem window
    whi: int       # last row of the subproblem window
    exact: bool = False   # window cut at the grid boundary: the operator's own profile

    @property
    def rows(self):
        return np.arange(self.lo, self.hi + 1)

    @property
    def w(self):
        return self.whi - self.wlo + 1


def _lower_window(lo, hi, b, k, full_window):
    """Window of a lower-front block with k buffer rows between the block and
    its moving PML (Sec. 2.2): [lo - k - b + 1, hi]; cut at row 1 when it
    would cross the boundary, where the window keeps the operator's own
    profile (an exact Schur inverse, as for the paper's first layers)."""
    if full_window:
        return Block("lower", lo, hi, 1, hi)
    wlo = lo - k - b + 1
    return Block("lower", lo, hi, max(wlo, 1), hi, exact=wlo < 1)


def _upper_window(lo, hi, b, k, n, full_window):
    if full_window:
        return Block("upper", lo, hi, lo, n)
    whi = hi + k + b - 1
    return Block("upper", lo, hi, lo, min(whi, n), exact=whi > n)


def partition_single(n, bp, b, dL, full_window=False, buffer=0):
    """Single-front partition of Sec. 2.1-2.2 (the formulation with a zero
    Dirichlet condition at x2 = 1 and the PML at x2 = 0 only): the front
    F = rows 1..bp, then blocks of d rows swept upward to the top row n, the
    last one taking the remainder (Algorithm 3 with d layers per step, Sec.
    2.3).  Every block's window is its rows plus b - 1 rows below; the top
    block's window ends at row n, next to the Dirichlet boundary.

    Returns (lower, [], None): the blocks in sweep order, no second front and
    no middle layer.
    """
    if n < bp + 1 or bp < 1 or dL < 1 or b < 1 or b > bp + 1:
        raise ValueError("invalid partition parameters")
    rows = n - bp
    sizes = [dL] * (rows // dL) + ([rows % dL] if rows % dL else [])
    lower = [Block("F", 1, bp, 1, bp)]
    lo = bp + 1
    for d in sizes:
        hi = lo + d - 1
        lower.append(_lower_window(lo, hi, b, buffer, full_window))
        lo = hi + 1
    return lower, [], None


def partition(n, bp, b, dL, full_window=False, buffer=0):
    """Two-front block partition of Sec. 2.3 (Fig. 2 left and right).

    The fronts sweep from F = rows 1..bp upward and from E = rows
    n-bp+1..n downward and meet at the middle layer (n+1)/2, which the paper
    visits last with moving PMLs on both sides.  Each front eliminates d
    rows per step; the rows between F and the middle layer number
    (n-1)/2 - bp, and when d does not divide them the last block of each
    front takes the remainder.

    Returns (lower, upper, middle): ``lower`` = [F, B_1, ..., B_K] in sweep
    order, ``upper`` = [E, B'_1, ..., B'_K], ``middle`` = the middle layer.
    With ``full_window`` every window extends to the domain boundary on its
    eliminated side (exact-limit test knob: then T~_B equals the exact Schur
    inverse, Sec. 2.2).  ``buffer`` = k rows between each block and its
    moving PML (Sec. 2.2, windows as in ``_lower_window``).
    """
    if n % 2 != 1 or n < 2 * bp + 1 or bp < 1 or dL < 1 or b < 1 or b > bp + 1:
        raise ValueError("invalid partition parameters")
    if (n + 1) // 2 - buffer - b < 0:
        raise ValueError("the middle layer's window does not fit")
    rows_front = (n - 1) // 2 - bp
    sizes = [dL] * (rows_front // dL) + ([rows_front % dL] if rows_front % dL else [])
    lower = [Block("F", 1, bp, 1, bp)]
    upper = [Block("E", n - bp + 1, n, n - bp + 1, n)]
    lo = bp + 1
    for d in sizes:
        hi = lo + d - 1
        lower.append(_lower_window(lo, hi, b, buffer, full_window))
        ulo, uhi = n + 1 - hi, n + 1 - lo
        upper.append(_upper_window(ulo, uhi, b, buffer, n, full_window))
        lo = hi + 1
    m = (n + 1) // 2
    if full_window:
        middle = Block("middle", m, m, 1, n)
    else:
        middle = Block("middle", m, m, m - buffer - b + 1, m + buffer + b - 1)
    return lower, upper, middle


def moving_sigma(t, eta_b, C):
    """One-sided quadratic profile (first branch of Eq. sigma) of width eta_b,
    zero for t >= eta_b; t is the distance from the window's Dirichlet row."""
    t = np.asarray(t, dtype=np.float64)
    out = np.zeros_like(t)
    m = t <= eta_b
    out[m] = (C / eta_b) * ((t[m] - eta_b) / eta_b) ** 2
    return out


def window_x2_stretch(blk, n, bp, b, C, omega, full_window=False, Cm=None, dirichlet_top=False):
    """x2 stretch of H_B on the window rows and at the half points.

    Returns (s_int, s_up, s_dn) of length w: s2 at rows wlo..whi, at (j+1/2)
    and at (j-1/2).  F, E and full-window blocks use the original boundary
    profile (strength C, part of A; one-sided sigma_2 for the Dirichlet-top
    formulation); moving blocks use the moving profile of Eq. helma with
    strength Cm (a parameter of the preconditioner only; None = C).
    """
    Cm = C if Cm is None else Cm
    h = 1.0 / (n + 1)
    j = np.arange(blk.wlo, blk.whi + 1, dtype=np.float64)
    if blk.kind in ("F", "E") or full_window or blk.exact:
        eta = bp * h
        prof = H.pml_sigma_one_sided if dirichlet_top else H.pml_sigma
        sig = lambda x: prof(x, eta, C)
    else:
        # the profile starts at the window's Dirichlet row(s) just outside it:
        # row lo - k - b below a lower block, hi + k + b above an upper one
        eta_b = b * h
        if blk.kind == "lower":
            d0 = blk.wlo - 1
            sig = lambda x: moving_sigma(x - d0 * h, eta_b, Cm)
        elif blk.kind == "upper":
            d1 = blk.whi + 1
            sig = lambda x: moving_sigma(d1 * h - x, eta_b, Cm)
        else:
            d0, d1 = blk.wlo - 1, blk.whi + 1
            sig = lambda x: moving_sigma(x - d0 * h, eta_b, Cm) + moving_sigma(d1 * h - x, eta_b, Cm)
    s_int = H.stretch(sig(j * h), omega)
    s_up = H.stretch(sig((j + 0.5) * h), omega)
    s_dn = H.stretch(sig((j - 0.5) * h), omega)
    return s_int, s_up, s_dn


def window_coefficients(blk, c, omega, bp, b, C, alpha, full_window=False, Cm=None, dirichlet_top=False):
    """Eq. helmd coefficients of H_B (Eq. helma discretised on the window)."""
    n = c.shape[0]
    h = 1.0 / (n + 1)
    s1 = H.axis_stretch(n, bp, C, omega)
    s_int, s_up, s_dn = window_x2_stretch(blk, n, bp, b, C, omega, full_window, Cm, dirichlet_top)
    rows = np.arange(blk.wlo, blk.whi + 1)
    return H.row_coefficients(c[rows - 1, :], omega, alpha, h, s1, s_int, s_up, s_dn)


def band_matrix_x2_first(coef):
    """LAPACK general-band storage of P_B H_B P_B^t (x2-first ordering).

    Unknown (i, j) of the window -> index (i-1) w + (j - wlo).  Half band
    width kl = ku = w.  Storage row kl + ku + r - s holds entry (r, s).
    """
    D = coef["D"]
    w, n = D.shape
    kl = ku = w
    Nw = w * n
    ab = np.zeros((2 * kl + ku + 1, Nw), dtype=np.complex128)

    def put(r, s, v):
        ab[kl + ku + r - s, s] = v

    idx = np.arange(Nw).reshape(n, w)           # idx[i-1, j-wlo]
    put(idx.ravel(), idx.ravel(), D.T.ravel())
    # x2 neighbours inside one x1 column: (j -> j+1) coefficient N, (j+1 -> j) S
    r = idx[:, :-1].ravel(); s = idx[:, 1:].ravel()
    put(r, s, coef["N"][:-1, :].T.ravel())
    put(s, r, coef["S"][1:, :].T.ravel())
    # x1 neighbours: (i -> i+1) coefficient E, (i+1 -> i) W
    r = idx[:-1, :].ravel(); s = idx[1:, :].ravel()
    put(r, s, coef["E"][:, :-1].T.ravel())
    put(s, r, coef["W"][:, 1:].T.ravel())
    return ab, kl, ku


@dataclass
class FactoredBlock:
    blk: Block
    lu: np.ndarray
    ipiv: np.ndarray
    kl: int
    ku: int
    n: int

    def t_tilde(self, g):
        """T~_B g: g has shape (R, d, n) on the block rows lo..hi; the
        right-hand side of H_B is zero on the other window rows (Eq. helma
        and the definition of T~ that follows it).  Returns (R, d, n)."""
        blk, n = self.blk, self.n
        w = blk.w
        R = g.shape[0]
        rhs = np.zeros((R, n, w), dtype=np.complex128)     # [r, i-1, j-wlo]
        off = blk.lo - blk.wlo
        rhs[:, :, off:off + (blk.hi - blk.lo + 1)] = np.transpose(g, (0, 2, 1))
        x, info = lapack.zgbtrs(self.lu, self.kl, self.ku, rhs.reshape(R, n * w).T, self.ipiv)
        if info != 0:
            raise RuntimeError("zgbtrs failed")
        x = x.T.reshape(R, n, w)
        return np.transpose(x[:, :, off:off + (blk.hi - blk.lo + 1)], (0, 2, 1)).copy()


def factor_block(blk, c, omega, bp, b, C, alpha, full_window=False, Cm=None, dirichlet_top=False):
    """One step of Algorithm 3: LU of P_B H_B P_B^t (LAPACK band LU)."""
    coef = window_coefficients(blk, c, omega, bp, b, C, alpha, full_window, Cm, dirichlet_top)
    ab, kl, ku = band_matrix_x2_first(coef)
    lu, ipiv, info = lapack.zgbtrf(ab, kl, ku)
    if info != 0:
        raise RuntimeError("zgbtrf: singular subproblem")
    return FactoredBlock(blk, lu, ipiv, kl, ku, c.shape[0])


@dataclass
class Setup:
    n: int
    lower: list
    upper: list
    middle: FactoredBlock
    Ncoup: np.ndarray      # N_{i,j} of A: coupling (i,j) -> (i,j+1), shape (n, n) [j-1, i-1]


def setup(c, omega, bp, b, dL, alpha, C, full_window=False, Cm=None, two_front=True, buffer=0):
    """Algorithm 3 (d layers per step): factor every block.  Cm: strength of
    the moving PMLs (None = C).  ``two_front`` False: the single-front
    Dirichlet-top formulation of Sec. 2.1-2.2 (one-sided sigma_2, one
    upward sweep, no middle layer).  ``buffer``: k rows between each block
    and its moving PML (Sec. 2.2)."""
    c = np.asarray(c, dtype=np.float64)
    n = c.shape[0]
    top = not two_front
    lower, upper, middle = (partition(n, bp, b, dL, full_window, buffer) if two_front
                            else partition_single(n, bp, b, dL, full_window, buffer))
    f = lambda blk: factor_block(blk, c, omega, bp, b, C, alpha, full_window, Cm, top)
    coef = H.stencil_coefficients(c, omega, bp, C, alpha, dirichlet_top=top)
    return Setup(n, [f(B) for B in lower], [f(B) for B in upper], f(middle) if middle is not None else None,
                 coef["N"])


def apply(st, r):
    """Algorithm 4 with two fronts (Sec. 2.3): u = M_alpha r.

    ``r`` has shape (R, n, n) or (n, n).  The couplings A_{m+1,m} are the
    x2 couplings of A (N_{i,m}; A and A_alpha share them).
    """
    squeeze = r.ndim == 2
    u = np.array(r, dtype=np.complex128).reshape((-1,) + r.shape[-2:]).copy()
    Nc = st.Ncoup
    rows = lambda B: slice(B.blk.lo - 1, B.blk.hi)
    v = {}
    n = st.n
    # forward sweep, lower front: u_{hi+1} -= A_{hi+1,hi} (T~_B u_B)_{hi}
    # (single front: the top block has no row above it)
    for k, B in enumerate(st.lower):
        v[k, 0] = B.t_tilde(u[:, rows(B), :])
        hi = B.blk.hi
        if hi < n:
            u[:, hi, :] -= Nc[hi - 1, :] * v[k, 0][:, -1, :]
    # forward sweep, upper front: u_{lo-1} -= A_{lo-1,lo} (T~_B u_B)_{lo}
    for k, B in enumerate(st.upper):
        v[k, 1] = B.t_tilde(u[:, rows(B), :])
        lo = B.blk.lo
        u[:, lo - 2, :] -= Nc[lo - 2, :] * v[k, 1][:, 0, :]
    # middle block with moving PMLs on both sides
    if st.middle is not None:
        u[:, rows(st.middle), :] = st.middle.t_tilde(u[:, rows(st.middle), :])
    # backward sweep, lower front: u_B = v_B - T~_B (A_{B,hi+1} u_{hi+1});
    # the single front's top block keeps u_B = v_B (Algorithm 4)
    for k in range(len(st.lower) - 1, -1, -1):
        B = st.lower[k]
        hi = B.blk.hi
        if hi == n:
            u[:, rows(B), :] = v[k, 0]
            continue
        g = np.zeros_like(v[k, 0])
        g[:, -1, :] = Nc[hi - 1, :] * u[:, hi, :]
        u[:, rows(B), :] = v[k, 0] - B.t_tilde(g)
    for k in range(len(st.upper) - 1, -1, -1):
        B = st.upper[k]
        lo = B.blk.lo
        g = np.zeros_like(v[k, 1])
        g[:, 0, :] = Nc[lo - 2, :] * u[:, lo - 2, :]
        u[:, rows(B), :] = v[k, 1] - B.t_tilde(g)
    return u[0] if squeeze else u


# ----------------------------------------------------------------------------
# Algorithms 1 and 2 with the same blocks: exact Schur complements (pin only).
# ----------------------------------------------------------------------------

def exact_setup(c, omega, bp, b, dL, alpha, C):
    """Algorithm 1 generalised to the two-front block order: dense
    T_B = S_B^{-1} with S_B = A_BB - A_{B,B-} T_{B-} A_{B-,B}.  Tiny n only."""
    c = np.asarray(c, dtype=np.float64)
    n = c.shape[0]
    A = H.helmholtz_matrix(c, omega, bp, C, alpha).toarray()
    lower, upper, middle = partition(n, bp, b, dL)
    idx = lambda B: np.arange((B.lo - 1) * n, B.hi * n)
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
    return dict(n=n, A=A, T=T, lower=lower, upper=upper, middle=middle)


def exact_apply(ex, f):
    """Algorithm 2 in the two-front block order: u = A^{-1} f exactly."""
    n, A, T = ex["n"], ex["A"], ex["T"]
    idx = lambda B: np.arange((B.lo - 1) * n, B.hi * n)
    u = np.array(f, dtype=np.complex128).reshape(-1).copy()
    for front in (ex["lower"], ex["upper"]):
        for k in range(len(front)):
            B = front[k]
            nxt = front[k + 1] if k + 1 < len(front) else ex["middle"]
            I, J = idx(B), idx(nxt)
            u[J] -= A[np.ix_(J, I)] @ (T[B.lo] @ u[I])
    for B in ex["lower"] + ex["upper"] + [ex["middle"]]:
        I = idx(B)
        u[I] = T[B.lo] @ u[I]
    for front in (ex["lower"], ex["upper"]):
        for k in range(len(front) - 1, -1, -1):
            B = front[k]
            nxt = front[k + 1] if k + 1 < len(front) else ex["middle"]
            I, J = idx(B), idx(nxt)
            u[I] -= T[B.lo] @ (A[np.ix_(I, J)] @ u[J])
    return u.reshape(n, n)


def exact_setup_single(c, omega, bp, b, dL, alpha, C):
    """Algorithm 1 in the single-front order of the Dirichlet-top formulation
    (Sec. 2.1): S_F = A_FF, S_m = A_mm - A_{m,m-1} T_{m-1} A_{m-1,m},
    T_m = S_m^{-1}, blocks of d rows upward to row n.  Tiny n only."""
    c = np.asarray(c, dtype=np.float64)
    n = c.shape[0]
    A = H.helmholtz_matrix(c, omega, bp, C, alpha, dirichlet_top=True).toarray()
    blocks, _, _ = partition_single(n, bp, b, dL)
    idx = lambda B: np.arange((B.lo - 1) * n, B.hi * n)
    T = []
    for k, B in enumerate(blocks):
        I = idx(B)
        S = A[np.ix_(I, I)].copy()
        if k > 0:
            P = idx(blocks[k - 1])
            S -= A[np.ix_(I, P)] @ T[k - 1] @ A[np.ix_(P, I)]
        T.append(np.linalg.inv(S))
    return dict(n=n, A=A, T=T, blocks=blocks)


def exact_apply_single(ex, f):
    """Algorithm 2 in the single-front order: u = A^{-1} f exactly."""
    n, A, T, blocks = ex["n"], ex["A"], ex["T"], ex["blocks"]
    idx = lambda B: np.arange((B.lo - 1) * n, B.hi * n)
    u = np.array(f, dtype=np.complex128).reshape(-1).copy()
    for k in range(len(blocks) - 1):
        I, J = idx(blocks[k]), idx(blocks[k + 1])
        u[J] -= A[np.ix_(J, I)] @ (T[k] @ u[I])
    for k, B in enumerate(blocks):
        I = idx(B)
        u[I] = T[k] @ u[I]
    for k in range(len(blocks) - 2, -1, -1):
        I, J = idx(blocks[k]), idx(blocks[k + 1])
        u[I] -= T[k] @ (A[np.ix_(I, J)] @ u[J])
    return u.reshape(n, n)
