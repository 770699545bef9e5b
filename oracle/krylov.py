"""Flexible GMRES with right preconditioning (Sec. 5.1: one V-cycle as the preconditioner).

FGMRES(m) (Saad's flexible variant): for j = 0..m-1
    z_j = M_j^{-1} v_j                           (one V-cycle)
    w   = A z_j
    h_{i,j} = (w, v_i), w -= h_{i,j} v_i          (modified Gram-Schmidt, i = 0..j,
                                                   then one re-orthogonalisation pass)
    h_{j+1,j} = ||w||,  v_{j+1} = w / h_{j+1,j}
    Givens rotations reduce H to triangular form; |g_{j+1}| is the residual norm estimate.
x = x_0 + Z_m y_m.  The iteration stops once the estimate is below rtol ||b||; the true
residual ||b - A x|| / ||b|| is then checked and the method restarts from x if needed.
Norms are Euclidean over the free DoFs (constrained slots are zero).

Pinned by: direct-solve parity on tiny grids and a one-iteration solve with the exact
preconditioner (tests/test_oracle_mg.py).
"""
from __future__ import annotations

import numpy as np


def fgmres(A, b: np.ndarray, precond, x0=None, rtol: float = 1e-8, restart: int = 50,
           maxit: int = 500):
    """Returns (x, info) with info = dict(iters, relres, converged, history)."""
    x = np.zeros_like(b) if x0 is None else x0.copy()
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return x, {"iters": 0, "relres": 0.0, "converged": True, "history": [0.0]}
    total = 0
    history = []
    while True:
        r = b - A @ x
        beta = np.linalg.norm(r)
        history.append(beta / bnorm)
        if beta <= rtol * bnorm or total >= maxit:
            return x, {"iters": total, "relres": beta / bnorm, "converged": beta <= rtol * bnorm,
                       "history": history}
        m = restart
        V = np.zeros((m + 1, b.size))
        Z = np.zeros((m, b.size))
        H = np.zeros((m + 1, m))
        cs = np.zeros(m)
        sn = np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        V[0] = r / beta
        k = 0
        for j in range(m):
            Z[j] = precond(V[j])
            w = A @ Z[j]
            for _pass in range(2):
                for i in range(j + 1):
                    hij = np.dot(w, V[i])
                    H[i, j] += hij
                    w = w - hij * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] != 0.0:
                V[j + 1] = w / H[j + 1, j]
            for i in range(j):                           # apply previous rotations
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
            total += 1
            history.append(abs(g[j + 1]) / bnorm)
            if abs(g[j + 1]) <= rtol * bnorm or total >= maxit:
                break
        y = np.zeros(k)
        for i in range(k - 1, -1, -1):                   # back substitution
            y[i] = (g[i] - np.dot(H[i, i + 1:k], y[i + 1:k])) / H[i, i]
        x = x + Z[:k].T @ y
