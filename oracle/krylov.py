"""Krylov solvers around the sweeping preconditioner (oracle; test infrastructure only).

Sec. 2.3 solves the preconditioned system M_alpha A u = M_alpha f with GMRES
(restart, initial guess and the precise residual are not stated; tolerance
1e-3 in the experiments).  Two forms are restated here, one RHS at a time:

* ``fgmres``: right-preconditioned flexible GMRES(m) (Saad's FGMRES):
  z_j = P(v_j), w = A z_j, modified Gram-Schmidt with one re-orthogonalisation
  pass, Givens rotations on the Hessenberg matrix, x = x0 + Z y; a restart
  recomputes the true residual f - A x.  Stops when ||f - A x|| <= tol ||f||.
* ``gmres_left``: GMRES(m) on M A u = M f with the preconditioned residual
  (the paper's formulation), stopping on ||M(f - A x)|| <= tol ||M f||.

Both are textbook Krylov methods; the tests pin them against a sparse direct
solve.
"""
import numpy as np


def _givens(a, b):
    """Complex Givens rotation (c real, s complex) with [c s; -conj(s) c] [a; b] = [r; 0]."""
    if b == 0:
        return 1.0, 0.0 + 0.0j
    if a == 0:
        return 0.0, np.conj(b) / abs(b)
    t = abs(a) + abs(b)
    na = t * np.sqrt(abs(a / t) ** 2 + abs(b / t) ** 2)
    c = abs(a) / na
    s = (a / abs(a)) * np.conj(b) / na
    return c, s


def fgmres(A, P, f, tol=1e-6, restart=30, maxit=500, x0=None):
    """Right-preconditioned flexible GMRES for one right-hand side.

    ``A`` and ``P`` are callables on 1-D complex vectors.  Returns
    (x, iterations, history of true relative residuals at restarts and of
    Givens estimates per iteration).
    """
    f = np.asarray(f, dtype=np.complex128).ravel()
    x = np.zeros_like(f) if x0 is None else np.array(x0, dtype=np.complex128).ravel()
    nf = np.linalg.norm(f)
    if nf == 0:
        return x, 0, [0.0]
    hist = []
    it = 0
    while True:
        r = f - A(x)
        beta = np.linalg.norm(r)
        hist.append(beta / nf)
        if beta <= tol * nf or it >= maxit:
            return x, it, hist
        m = restart
        V = [r / beta]
        Z = []
        Hm = np.zeros((m + 1, m), dtype=np.complex128)
        cs = np.zeros(m)
        sn = np.zeros(m, dtype=np.complex128)
        g = np.zeros(m + 1, dtype=np.complex128)
        g[0] = beta
        k = 0
        for j in range(m):
            z = P(V[j])
            Z.append(z)
            w = A(z)
            for _ in range(2):                          # MGS + one re-orthogonalisation
                for i in range(j + 1):
                    hij = np.vdot(V[i], w)
                    Hm[i, j] += hij
                    w = w - hij * V[i]
            Hm[j + 1, j] = np.linalg.norm(w)
            V.append(w / Hm[j + 1, j] if Hm[j + 1, j] != 0 else w)
            for i in range(j):                          # apply previous rotations
                t = cs[i] * Hm[i, j] + sn[i] * Hm[i + 1, j]
                Hm[i + 1, j] = -np.conj(sn[i]) * Hm[i, j] + cs[i] * Hm[i + 1, j]
                Hm[i, j] = t
            cs[j], sn[j] = _givens(Hm[j, j], Hm[j + 1, j])
            Hm[j, j] = cs[j] * Hm[j, j] + sn[j] * Hm[j + 1, j]
            Hm[j + 1, j] = 0.0
            g[j + 1] = -np.conj(sn[j]) * g[j]
            g[j] = cs[j] * g[j]
            it += 1
            k = j + 1
            hist.append(abs(g[j + 1]) / nf)
            if abs(g[j + 1]) <= tol * nf or it >= maxit:
                break
        y = np.linalg.solve(np.triu(Hm[:k, :k]), g[:k])
        for i in range(k):
            x = x + y[i] * Z[i]


def gmres_left(A, M, f, tol=1e-3, restart=30, maxit=500):
    """GMRES(m) on M A u = M f (Sec. 2.3), preconditioned-residual stopping."""
    f = np.asarray(f, dtype=np.complex128).ravel()
    x = np.zeros_like(f)
    Mf = M(f)
    nMf = np.linalg.norm(Mf)
    it = 0
    hist = []
    while True:
        r = M(f - A(x))
        beta = np.linalg.norm(r)
        hist.append(beta / nMf)
        if beta <= tol * nMf or it >= maxit:
            return x, it, hist
        m = restart
        V = [r / beta]
        Hm = np.zeros((m + 1, m), dtype=np.complex128)
        cs = np.zeros(m)
        sn = np.zeros(m, dtype=np.complex128)
        g = np.zeros(m + 1, dtype=np.complex128)
        g[0] = beta
        k = 0
        for j in range(m):
            w = M(A(V[j]))
            for _ in range(2):
                for i in range(j + 1):
                    hij = np.vdot(V[i], w)
                    Hm[i, j] += hij
                    w = w - hij * V[i]
            Hm[j + 1, j] = np.linalg.norm(w)
            V.append(w / Hm[j + 1, j] if Hm[j + 1, j] != 0 else w)
            for i in range(j):
                t = cs[i] * Hm[i, j] + sn[i] * Hm[i + 1, j]
                Hm[i + 1, j] = -np.conj(sn[i]) * Hm[i, j] + cs[i] * Hm[i + 1, j]
                Hm[i, j] = t
            cs[j], sn[j] = _givens(Hm[j, j], Hm[j + 1, j])
            Hm[j, j] = cs[j] * Hm[j, j] + sn[j] * Hm[j + 1, j]
            Hm[j + 1, j] = 0.0
            g[j + 1] = -np.conj(sn[j]) * g[j]
            g[j] = cs[j] * g[j]
            it += 1
            k = j + 1
            hist.append(abs(g[j + 1]) / nMf)
            if abs(g[j + 1]) <= tol * nMf or it >= maxit:
                break
        y = np.linalg.solve(np.triu(Hm[:k, :k]), g[:k])
        x = x + np.array(V[:k]).T @ y
