"""Steady manufactured problem of Sec. 5.1 (used for the convergence-rate and Table 4 pins).

Exact solution (Sec. 5.1):  u = curl phi = (d phi/dy, -d phi/dx),  phi = [x y (1-x)(1-y)]^2,
p = 1,  w = 0.  Since div u = 0 and p is constant, the loads are rho g = -mu Laplace(u),
rho_f g = 0 and, for the single backward-Euler step from the exact state, the P0 load is
(1/M) p, i.e. the right-hand side row of a triangle is -(1/M)|T|.  The pressure condition
is natural: p = 1 on the boundary enters the RT0 rows as -tau <p, psi . n_out>.

Load integrals use Radon's 7-point degree-5 rule on each triangle.  Pinned by
tests/test_oracle_manufactured.py (the exact field against symbolic derivatives of phi, its
divergence and boundary values, the rule's exactness to degree 5, the load vector's P0 and
boundary rows) and through the convergence rates the paper states (first order for |u|_H1,
second order for ||p||_L2, Sec. 5.1) in tests/test_oracle_mg.py.
"""
from __future__ import annotations

import numpy as np

from .fem import Params, Triangle, reference_triangles
from .mesh import Mesh

_S15 = np.sqrt(15.0)
_A = (6.0 - _S15) / 21.0
_B = (6.0 + _S15) / 21.0
RADON_BARY = np.array([[1 / 3, 1 / 3, 1 / 3],
                       [_A, _A, 1 - 2 * _A], [_A, 1 - 2 * _A, _A], [1 - 2 * _A, _A, _A],
                       [_B, _B, 1 - 2 * _B], [_B, 1 - 2 * _B, _B], [1 - 2 * _B, _B, _B]])
RADON_W = np.array([9 / 40] + [(155 - _S15) / 1200] * 3 + [(155 + _S15) / 1200] * 3)


def _F(x):
    X, dX = x * (1 - x), 1 - 2 * x
    return X * X, 2 * X * dX, 2 * dX * dX - 4 * X, -12 * dX      # F, F', F'', F'''


def exact_u(x, y):
    F, F1, _, _ = _F(x)
    G, G1, _, _ = _F(y)
    return np.array([F * G1, -F1 * G])


def exact_grad_u(x, y):
    """Rows: components; columns: d/dx, d/dy."""
    F, F1, F2, _ = _F(x)
    G, G1, G2, _ = _F(y)
    return np.array([[F1 * G1, F * G2], [-F2 * G, -F1 * G1]])


def body_force(x, y, mu):
    """rho g = -mu Laplace(u) for the divergence-free exact displacement."""
    F, F1, F2, F3 = _F(x)
    G, G1, G2, G3 = _F(y)
    lap = np.array([F2 * G1 + F * G3, -(F3 * G + F1 * G2)])
    return -mu * lap


def rhs(mesh: Mesh, prm: Params) -> np.ndarray:
    n, h = mesh.n, mesh.h
    b = np.zeros(mesh.ndof)
    for o, i, j in mesh.triangles():
        X = np.array(Mesh.tri_vertices(o, i, j), dtype=float) * h
        t = Triangle(X, [e[0] for e in Mesh.tri_edges(o, i, j)])
        dofs = mesh.tri_dofs(o, i, j)
        for lam, wq in zip(RADON_BARY, RADON_W):
            x = lam @ t.X
            f = body_force(x[0], x[1], prm.mu)
            vals, _ = t.u_basis(x)
            b[dofs[:9]] += wq * t.area * (vals @ f)
        b[dofs[12]] += -prm.inv_M * t.area * 1.0
    # natural pressure condition p = 1 on the boundary: -tau <p, psi_e . n_out>
    for i in range(n):
        b[mesh.idx("wh", i, 0)] += -prm.tau * h * (-1.0)     # bottom: n_out = -n_h
        b[mesh.idx("wh", i, n)] += -prm.tau * h * (+1.0)     # top:    n_out = +n_h
    for j in range(n):
        b[mesh.idx("wv", 0, j)] += -prm.tau * h * (-1.0)     # left:   n_out = -n_v
        b[mesh.idx("wv", n, j)] += -prm.tau * h * (+1.0)     # right:  n_out = +n_v
    return b * mesh.free


def errors(mesh: Mesh, x: np.ndarray):
    """(|u - u_h|_H1, ||p - p_h||_L2) with the 7-point rule for the displacement."""
    h = mesh.h
    e_u = 0.0
    e_p = 0.0
    for o, i, j in mesh.triangles():
        X = np.array(Mesh.tri_vertices(o, i, j), dtype=float) * h
        t = Triangle(X, [e[0] for e in Mesh.tri_edges(o, i, j)])
        dofs = mesh.tri_dofs(o, i, j)
        coef = x[dofs[:9]]
        for lam, wq in zip(RADON_BARY, RADON_W):
            xq = lam @ t.X
            _, G = t.u_basis(xq)
            gh = np.einsum("a,acs->cs", coef, G)
            d = exact_grad_u(xq[0], xq[1]) - gh
            e_u += wq * t.area * float(np.sum(d * d))
        e_p += t.area * (1.0 - x[dofs[12]]) ** 2
    return np.sqrt(e_u), np.sqrt(e_p)
