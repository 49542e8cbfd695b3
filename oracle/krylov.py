"""Right-preconditioned GMRES with modified Gram-Schmidt and Givens rotations.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Sect. 4: PGMRES stops when the residual norm falls below the tolerance or
after 300 iterations.  Reading: right preconditioning, x0 = 0, the test is
on the relative residual of the unpreconditioned system ||b - A x|| / ||b||
(which right preconditioning leaves as the quantity GMRES minimises).  An
iteration is one Arnoldi step (one product with A and one with M^{-1}).
"""
from __future__ import annotations

import numpy as np


def gmres(A, b, M=None, rtol=1e-8, restart=0, max_iter=300):
    """Solve A x = b.  A, M are callables.  restart=0 means no restart."""
    M = M or (lambda v: v)
    n = b.shape[0]
    bnorm = float(np.linalg.norm(b))
    x = np.zeros(n)
    hist = [1.0]
    if bnorm == 0.0:
        return x, dict(iters=0, relres=0.0, history=hist, converged=True)
    m = max_iter if restart <= 0 else restart
    its = 0
    r = b.copy()
    converged = False
    while its < max_iter:
        beta = float(np.linalg.norm(r))
        if beta <= rtol * bnorm:
            converged = True
            break
        V = np.zeros((m + 1, n))
        H = np.zeros((m + 1, m))
        cs, sn = np.zeros(m), np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        V[0] = r / beta
        k = 0
        for j in range(m):
            if its >= max_iter:
                break
            w = A(M(V[j]))
            for i in range(j + 1):
                H[i, j] = w @ V[i]
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] > 0:
                V[j + 1] = w / H[j + 1, j]
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            den = np.hypot(H[j, j], H[j + 1, j])
            cs[j], sn[j] = H[j, j] / den, H[j + 1, j] / den
            H[j, j] = den
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            its += 1
            k = j + 1
            hist.append(abs(g[j + 1]) / bnorm)
            if abs(g[j + 1]) <= rtol * bnorm:
                converged = True
                break
        y = np.linalg.solve(np.triu(H[:k, :k]), g[:k]) if k else np.zeros(0)
        x = x + M(V[:k].T @ y)
        r = b - A(x)
        if converged:
            break
    relres = float(np.linalg.norm(b - A(x)) / bnorm)
    return x, dict(iters=its, relres=relres, history=hist, converged=converged)
