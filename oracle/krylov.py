"""Flexible GMRES of the oracle (outer Krylov solver of Sec. 3 and Sec. 5), plain numpy.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Right-preconditioned FGMRES(m) (Saad, SIAM J. Sci. Comput. 14, 1993) with modified
Gram-Schmidt Arnoldi and Givens rotations.  Stops when the Arnoldi residual estimate drops to
rtol * ||b - A x0||; at each restart the true residual is recomputed.
"""
from __future__ import annotations

import numpy as np


def fgmres(apply_A, b, precond, x0=None, rtol=1e-8, restart=30, maxit=500):
    n = b.shape[0]
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64)
    r = b - apply_A(x)
    beta0 = float(np.linalg.norm(r))
    target = rtol * beta0
    its = 0
    history = [beta0]
    while True:
        r = b - apply_A(x)
        beta = float(np.linalg.norm(r))
        if beta <= target or its >= maxit or beta == 0.0:
            break
        V = np.zeros((restart + 1, n))
        Z = np.zeros((restart, n))
        H = np.zeros((restart + 1, restart))
        cs = np.zeros(restart)
        sn = np.zeros(restart)
        g = np.zeros(restart + 1)
        g[0] = beta
        V[0] = r / beta
        k = 0
        for j in range(restart):
            Z[j] = precond(V[j])
            w = apply_A(Z[j])
            for i in range(j + 1):
                H[i, j] = float(w @ V[i])
                w = w - H[i, j] * V[i]
            H[j + 1, j] = float(np.linalg.norm(w))
            if H[j + 1, j] > 0.0:
                V[j + 1] = w / H[j + 1, j]
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            den = float(np.hypot(H[j, j], H[j + 1, j]))
            cs[j] = H[j, j] / den
            sn[j] = H[j + 1, j] / den
            H[j, j] = den
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            its += 1
            k = j + 1
            history.append(abs(g[j + 1]))
            if abs(g[j + 1]) <= target or its >= maxit:
                break
        y = np.zeros(k)
        for i in range(k - 1, -1, -1):
            y[i] = (g[i] - H[i, i + 1:k] @ y[i + 1:k]) / H[i, i]
        x = x + Z[:k].T @ y
    r = b - apply_A(x)
    return x, its, float(np.linalg.norm(r)), beta0, history
