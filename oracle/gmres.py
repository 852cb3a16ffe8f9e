"""Oracle: plain restarted GMRES -- TEST INFRASTRUCTURE ONLY.

The paper solves A sigma_b = b with GMRES in matrix-free form: only the action
A sigma is supplied (Sec. III, electrostatic implementation; Sec. IV.B uses a
relative tolerance of 1e-5).  This is restarted GMRES(m) of Saad & Schultz
(1986): Arnoldi with modified Gram-Schmidt, Givens rotations on the Hessenberg
matrix, stop when the rotated residual |g_{k+1}| <= tol * ||b||, then the
triangular solve and the update x += V y.  Everything is FP64 numpy.
"""
from __future__ import annotations

import numpy as np


def gmres(matvec, b, x0=None, tol=1e-6, restart=50, max_iter=1000):
    """Return (x, iterations, relative residual estimate, converged)."""
    b = np.asarray(b, dtype=np.float64)
    n = b.size
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64)
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return np.zeros(n), 0, 0.0, True
    it = 0
    rel = np.inf
    while it < max_iter:
        r = b - matvec(x)
        beta = np.linalg.norm(r)
        rel = beta / bnorm
        if rel <= tol:
            return x, it, rel, True
        m = min(restart, max_iter - it)
        V = np.zeros((m + 1, n))
        H = np.zeros((m + 1, m))
        cs = np.zeros(m)
        sn = np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        V[0] = r / beta
        k_done = 0
        for k in range(m):
            w = matvec(V[k])
            for i in range(k + 1):          # modified Gram-Schmidt
                H[i, k] = np.dot(w, V[i])
                w = w - H[i, k] * V[i]
            H[k + 1, k] = np.linalg.norm(w)
            if H[k + 1, k] > 0.0:
                V[k + 1] = w / H[k + 1, k]
            for i in range(k):              # earlier rotations on the new column
                t = cs[i] * H[i, k] + sn[i] * H[i + 1, k]
                H[i + 1, k] = -sn[i] * H[i, k] + cs[i] * H[i + 1, k]
                H[i, k] = t
            den = np.hypot(H[k, k], H[k + 1, k])
            cs[k], sn[k] = H[k, k] / den, H[k + 1, k] / den
            H[k, k] = den
            H[k + 1, k] = 0.0
            g[k + 1] = -sn[k] * g[k]
            g[k] = cs[k] * g[k]
            it += 1
            k_done = k + 1
            rel = abs(g[k + 1]) / bnorm
            if rel <= tol or H[k, k] == 0.0:
                break
        y = np.zeros(k_done)
        for i in range(k_done - 1, -1, -1):  # back substitution
            y[i] = (g[i] - np.dot(H[i, i + 1:k_done], y[i + 1:k_done])) / H[i, i]
        x = x + V[:k_done].T @ y
        if rel <= tol:
            return x, it, rel, True
    return x, it, rel, False
