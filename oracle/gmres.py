"""Restarted GMRES (Saad and Schultz 1986), as used for Eq. (AEFIEoutJ) (Sec. III-E: the solver
needs only products with the system matrix). Test infrastructure (oracle), FP64.

Modified Gram-Schmidt Arnoldi, Givens rotations on the Hessenberg matrix, restart length m,
stopping on the relative residual ||b - A x|| / ||b|| (the recurrence's estimate; the caller
verifies with a true residual). An optional right preconditioner M (x = M u) may vary between
iterations (flexible GMRES): the preconditioned directions Z are then kept.
"""
from __future__ import annotations

import numpy as np


def gmres(matvec, b, tol=1e-6, restart=100, max_iter=2000, x0=None, precond=None):
    b = np.asarray(b, dtype=np.complex128)
    n = b.size
    x = np.zeros(n, dtype=np.complex128) if x0 is None else np.array(x0, dtype=np.complex128)
    bnorm = np.linalg.norm(b)
    if bnorm == 0:
        return x, 0, [0.0]
    hist = []
    it = 0
    while it < max_iter:
        r = b - matvec(x)
        beta = np.linalg.norm(r)
        hist.append(beta / bnorm)
        if beta / bnorm <= tol:
            return x, it, hist
        m = min(restart, max_iter - it)
        V = np.zeros((m + 1, n), dtype=np.complex128)
        Zd = np.zeros((m, n), dtype=np.complex128) if precond is not None else None
        H = np.zeros((m + 1, m), dtype=np.complex128)
        cs = np.zeros(m, dtype=np.complex128)
        sn = np.zeros(m, dtype=np.complex128)
        g = np.zeros(m + 1, dtype=np.complex128)
        g[0] = beta
        V[0] = r / beta
        k_done = 0
        for k in range(m):
            z = precond(V[k]) if precond is not None else V[k]
            if Zd is not None:
                Zd[k] = z
            w = matvec(z)
            for i in range(k + 1):
                H[i, k] = np.vdot(V[i], w)
                w = w - H[i, k] * V[i]
            H[k + 1, k] = np.linalg.norm(w)
            if H[k + 1, k] != 0:
                V[k + 1] = w / H[k + 1, k]
            # complex Givens rotation (c, s) acting as (x, y) -> (conj(c) x + conj(s) y, -s x + c y)
            for i in range(k):
                t = np.conj(cs[i]) * H[i, k] + np.conj(sn[i]) * H[i + 1, k]
                H[i + 1, k] = -sn[i] * H[i, k] + cs[i] * H[i + 1, k]
                H[i, k] = t
            a, bb = H[k, k], H[k + 1, k]
            den = np.sqrt(abs(a) ** 2 + abs(bb) ** 2)
            cs[k] = a / den if den != 0 else 1.0
            sn[k] = bb / den if den != 0 else 0.0
            H[k, k] = den
            H[k + 1, k] = 0.0
            g[k + 1] = -sn[k] * g[k]
            g[k] = np.conj(cs[k]) * g[k]
            it += 1
            k_done = k + 1
            hist.append(abs(g[k + 1]) / bnorm)
            if abs(g[k + 1]) / bnorm <= tol:
                break
        y = np.linalg.solve(np.triu(H[:k_done, :k_done]), g[:k_done])
        D = Zd[:k_done] if Zd is not None else V[:k_done]
        x = x + D.T @ y
        if hist[-1] <= tol:
            r = b - matvec(x)
            hist.append(np.linalg.norm(r) / bnorm)
            if hist[-1] <= tol:
                return x, it, hist
    return x, it, hist
