"""Restarted flexible GMRES (right preconditioning) with modified Gram-Schmidt, FP64.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The paper (Section 3) solves each linearised system with a restarted FGMRES method
preconditioned by the multilevel overlapping Schwarz operator; it gives no further
details, so this is the textbook algorithm (Saad's flexible GMRES): Arnoldi on
A z_j with z_j = B v_j, Givens rotations for the Hessenberg least-squares problem,
x = x0 + Z y at the end of a cycle, stop when ||b - A x|| / ||b|| <= tol (checked on the
true residual at the end of every cycle).

Parity status: pinned (least-squares optimality against a dense solve on small cases).
"""
from __future__ import annotations

import numpy as np


def fgmres(A, b, M, tol=1e-8, restart=100, max_it=1000, x0=None, keep_basis=False):
    """Solve A x = b.  A, M: callables (matvec, preconditioner apply).

    Returns x, info dict(iterations, relres (true), history (estimated residual ratios),
    converged, and the last cycle's Z, V, H if keep_basis)."""
    n = b.size
    x = np.zeros(n) if x0 is None else x0.copy()
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return x, dict(iterations=0, relres=0.0, history=[0.0], converged=True)
    it = 0
    hist = []
    r = b - A(x)
    beta = np.linalg.norm(r)
    hist.append(beta / bnorm)
    info = {}
    while it < max_it and beta / bnorm > tol:
        m = min(restart, max_it - it)
        V = np.zeros((m + 1, n))
        Z = np.zeros((m, n))
        H = np.zeros((m + 1, m))
        cs = np.zeros(m)
        sn = np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        V[0] = r / beta
        j_done = 0
        for j in range(m):
            Z[j] = M(V[j])
            w = A(Z[j])
            for i in range(j + 1):               # modified Gram-Schmidt
                H[i, j] = V[i] @ w
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] != 0.0:
                V[j + 1] = w / H[j + 1, j]
            for i in range(j):                    # apply previous rotations
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            den = np.hypot(H[j, j], H[j + 1, j])
            cs[j], sn[j] = H[j, j] / den, H[j + 1, j] / den
            H[j, j] = den
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            it += 1
            j_done = j + 1
            hist.append(abs(g[j + 1]) / bnorm)
            if abs(g[j + 1]) / bnorm <= tol:
                break
        y = np.linalg.solve(np.triu(H[:j_done, :j_done]), g[:j_done])
        x = x + Z[:j_done].T @ y
        r = b - A(x)
        beta = np.linalg.norm(r)
        if keep_basis:
            info = dict(Z=Z[:j_done].copy(), V=V[:j_done + 1].copy(), y=y)
    res = np.linalg.norm(b - A(x)) / bnorm
    info.update(iterations=it, relres=res, history=hist, converged=res <= tol)
    return x, info
