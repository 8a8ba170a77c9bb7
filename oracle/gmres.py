"""Dense GMRES (Sec. 3.3: K Phi = b solved by GMRES to a relative tolerance, Sec. 5).

Test infrastructure only: used by tests/, the smoke check and bench.py's CPU
baseline; the library never imports or calls it.

Plain textbook GMRES: Arnoldi with modified Gram-Schmidt, Givens rotations
for the Hessenberg least-squares problem, x0 = 0, no restart, optional RIGHT
preconditioner M (so that the monitored residual is the true residual
||b - K Phi|| / ||b|| of the unpreconditioned system).
"""

from __future__ import annotations

import numpy as np


def gmres(matvec, b, tol: float = 1e-8, maxiter: int = 1000, M=None):
    """Return (x, iterations, residual history (relative), converged)."""
    b = np.asarray(b, dtype=np.complex128)
    n = b.size
    beta = np.linalg.norm(b)
    if beta == 0.0:
        return np.zeros(n, dtype=np.complex128), 0, [0.0], True
    m = min(maxiter, n)
    V = np.zeros((n, m + 1), dtype=np.complex128)
    H = np.zeros((m + 1, m), dtype=np.complex128)
    cs = np.zeros(m, dtype=np.complex128)
    sn = np.zeros(m, dtype=np.complex128)
    g = np.zeros(m + 1, dtype=np.complex128)
    g[0] = beta
    V[:, 0] = b / beta
    hist = [1.0]
    j_done = 0
    for j in range(m):
        z = M(V[:, j]) if M is not None else V[:, j]
        w = matvec(z)
        for i in range(j + 1):  # modified Gram-Schmidt
            H[i, j] = np.vdot(V[:, i], w)
            w = w - H[i, j] * V[:, i]
        H[j + 1, j] = np.linalg.norm(w)
        if H[j + 1, j] != 0:
            V[:, j + 1] = w / H[j + 1, j]
        for i in range(j):  # apply previous rotations
            t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
            H[i + 1, j] = -np.conj(sn[i]) * H[i, j] + np.conj(cs[i]) * H[i + 1, j]
            H[i, j] = t
        a, c = H[j, j], H[j + 1, j]
        r = np.hypot(abs(a), abs(c))
        if r == 0:
            cs[j], sn[j] = 1.0, 0.0
        elif a == 0:
            cs[j], sn[j] = 0.0, np.conj(c) / abs(c)
        else:
            cs[j] = abs(a) / r
            sn[j] = (a / abs(a)) * np.conj(c) / r
        H[j, j] = cs[j] * a + sn[j] * c
        H[j + 1, j] = 0.0
        g[j + 1] = -np.conj(sn[j]) * g[j]
        g[j] = cs[j] * g[j]
        j_done = j + 1
        res = abs(g[j + 1]) / beta
        hist.append(res)
        if res <= tol:
            break
    y = np.linalg.solve(np.triu(H[:j_done, :j_done]), g[:j_done])
    x = V[:, :j_done] @ y
    if M is not None:
        x = M(x)
    return x, j_done, hist, hist[-1] <= tol
