"""Restarted GMRES, plain FP64 (Sec. 4: matrix-free GMRES, one operator apply per iteration).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Modified Gram-Schmidt Arnoldi, Givens rotations on the Hessenberg matrix, restart
length m. The Givens residual estimate decides when a cycle stops; the true residual
b - A x is recomputed at the end of every cycle and decides convergence.
"""
from __future__ import annotations

import numpy as np


def gmres(matvec, b, x0=None, tol=1e-10, restart=100, max_iter=1000):
    """Solve A x = b. Returns (x, info) with info = dict(iterations, restarts, rel_residual, converged)."""
    b = np.asarray(b, dtype=np.float64)
    n = b.shape[0]
    m = min(restart, n)
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64)
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return np.zeros(n), dict(iterations=0, restarts=0, rel_residual=0.0, converged=True)
    r = b - matvec(x) if np.any(x) else b.copy()
    beta = np.linalg.norm(r)
    its = 0
    cycles = 0
    while beta > tol * bnorm and its < max_iter:
        V = np.zeros((m + 1, n))
        H = np.zeros((m + 1, m))
        cs = np.zeros(m)
        sn = np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        V[0] = r / beta
        k = 0
        for j in range(m):
            w = matvec(V[j])
            its += 1
            for i in range(j + 1):
                H[i, j] = np.dot(w, V[i])
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            breakdown = H[j + 1, j] == 0.0
            if not breakdown:
                V[j + 1] = w / H[j + 1, j]
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            den = np.hypot(H[j, j], H[j + 1, j])
            cs[j] = H[j, j] / den
            sn[j] = H[j + 1, j] / den
            H[j, j] = den
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            k = j + 1
            if abs(g[j + 1]) <= tol * bnorm or its >= max_iter or breakdown:
                break
        y = np.zeros(k)
        for i in range(k - 1, -1, -1):
            y[i] = (g[i] - np.dot(H[i, i + 1:k], y[i + 1:k])) / H[i, i]
        x = x + V[:k].T @ y
        r = b - matvec(x)
        beta = np.linalg.norm(r)
        cycles += 1
    rel = beta / bnorm
    return x, dict(iterations=its, restarts=max(cycles - 1, 0), rel_residual=rel, converged=rel <= tol)
