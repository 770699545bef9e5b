"""Backward-Euler time stepping of Biot's model (Sec. 2.1, Eqs. discrete1-3) on a smooth
time-dependent manufactured solution (in the spirit of Sec. 5.2's smooth test problem).

Test infrastructure: the oracle of the library's time-stepping entry point
(bmg_backward_euler_rhs) and of its time loop.

Exact solution (the smooth problem of Sec. 5.2 has non-zero boundary displacement; the
reading used here keeps the library's boundary conditions, displacement zero and pressure
natural with zero data):
    u = e^{-t} curl phi,  phi = [x y (1-x)(1-y)]^2      (Sec. 5.1's field; u = 0 on the boundary)
    p = e^{-t} sin(pi x) sin(pi y)                       (p = 0 on the boundary)
    w = -K grad p.
Loads of Biot's equations (Sec. 2): div u = 0, so the lambda term drops out and
    rho g   = e^{-t} (-mu Laplace(curl phi)) + alpha grad p,
    rho_f g = 0                                         (K^{-1} w + grad p = 0),
    f       = (1/M) dp/dt + alpha d(div u)/dt + div w = (2 pi^2 K - 1/M) p.
Step m (t_m = m tau), with eq. discrete3 scaled by -1:
    A x^m = load(t_m) + history(x^{m-1}),
    load:    u rows (rho g(t_m), v),  w rows 0,  p rows -tau (f(t_m), q);
    history: p rows alpha B_u u^{m-1} - (1/M) M_p p^{m-1}, the p rows of A applied to
             (u^{m-1}, 0, p^{m-1}).
Initial state x^0 = (0, 0, cell averages of p(0)), whose history term is the exact
alpha (div u(0), q) - (1/M) (p(0), q) (div u(0) = 0).  Integrals use Radon's 7-point rule.

Pinned by: the loads against symbolic derivatives of the exact fields, and first-order
(|u|_H1) and second-order (p against its cell averages) convergence of the final-time
errors with tau = h^2 (tests/test_oracle_timedep.py).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse.linalg as spla

from . import fem
from .fem import Params, Triangle
from .manufactured import RADON_BARY, RADON_W, body_force, exact_grad_u
from .mesh import Mesh


def exact_p(x, y, t):
    return np.exp(-t) * np.sin(np.pi * x) * np.sin(np.pi * y)


def grad_p(x, y, t):
    e = np.exp(-t) * np.pi
    return np.array([e * np.cos(np.pi * x) * np.sin(np.pi * y), e * np.sin(np.pi * x) * np.cos(np.pi * y)])


def source_f(x, y, t, prm: Params, K: float):
    """f = (1/M) dp/dt + div w = (2 pi^2 K - 1/M) p."""
    return (2.0 * np.pi ** 2 * K - prm.inv_M) * exact_p(x, y, t)


def u_force(x, y, t, prm: Params):
    """rho g = e^{-t} (-mu Laplace(curl phi)) + alpha grad p."""
    return np.exp(-t) * body_force(x, y, prm.mu) + prm.alpha * grad_p(x, y, t)


def _triangles(mesh: Mesh):
    h = mesh.h
    for o, i, j in mesh.triangles():
        X = np.array(Mesh.tri_vertices(o, i, j), dtype=float) * h
        yield o, i, j, Triangle(X, [e[0] for e in Mesh.tri_edges(o, i, j)])


def loads(mesh: Mesh, prm: Params, K: float, t: float) -> np.ndarray:
    """The step's load vector at time t (u rows, zero w rows, -tau (f, q) p rows)."""
    b = np.zeros(mesh.ndof)
    for o, i, j, tri in _triangles(mesh):
        dofs = mesh.tri_dofs(o, i, j)
        for lam, wq in zip(RADON_BARY, RADON_W):
            x = lam @ tri.X
            vals, _ = tri.u_basis(x)
            b[dofs[:9]] += wq * tri.area * (vals @ u_force(x[0], x[1], t, prm))
            b[dofs[12]] += -prm.tau * wq * tri.area * source_f(x[0], x[1], t, prm, K)
    return b * mesh.free


def cell_averages_p(mesh: Mesh, t: float) -> np.ndarray:
    """Vector with the cell averages of p(t) in the P0 slots and zero elsewhere."""
    x = np.zeros(mesh.ndof)
    for o, i, j, tri in _triangles(mesh):
        dofs = mesh.tri_dofs(o, i, j)
        x[dofs[12]] = sum(wq * exact_p(*(lam @ tri.X), t) for lam, wq in zip(RADON_BARY, RADON_W))
    return x


def history(A, mesh: Mesh, x_prev: np.ndarray) -> np.ndarray:
    """p rows of A applied to (u_prev, 0, p_prev); zero in the u and w rows."""
    pm = fem.type_mask(mesh, fem.P_TYPES)
    wm = fem.type_mask(mesh, fem.W_TYPES)
    return np.where(pm, A @ np.where(wm, 0.0, x_prev), 0.0)


def errors(mesh: Mesh, x: np.ndarray, t: float):
    """(|u(t) - u_h|_H1, ||Pi_0 p(t) - p_h||_L2): the displacement error with the 7-point rule,
    the pressure against its cell averages."""
    e_u = e_p = 0.0
    avg = cell_averages_p(mesh, t)
    for o, i, j, tri in _triangles(mesh):
        dofs = mesh.tri_dofs(o, i, j)
        coef = x[dofs[:9]]
        for lam, wq in zip(RADON_BARY, RADON_W):
            xq = lam @ tri.X
            _, G = tri.u_basis(xq)
            d = np.exp(-t) * exact_grad_u(xq[0], xq[1]) - np.einsum("a,acs->cs", coef, G)
            e_u += wq * tri.area * float(np.sum(d * d))
        e_p += tri.area * (avg[dofs[12]] - x[dofs[12]]) ** 2
    return np.sqrt(e_u), np.sqrt(e_p)


def run(n: int, prm: Params, K: float, steps: int, solve=None):
    """``steps`` backward-Euler steps of size prm.tau from x^0 on an n-cell grid with uniform
    permeability K.  ``solve(A, b, x_guess)`` defaults to a direct sparse solve on the free
    DoFs (A is factored once).  Returns (mesh, A, list of x^m for m = 0..steps)."""
    mesh = Mesh(n)
    kinv = np.full((n, n), 1.0 / K)
    A = fem.assemble(mesh, prm, kinv, kinv)
    fi = mesh.free_idx
    if solve is None:
        lu = spla.splu(A[fi][:, fi].tocsc())

        def solve(A_, b, x_guess):
            x = np.zeros_like(b)
            x[fi] = lu.solve(b[fi])
            return x
    xs = [cell_averages_p(mesh, 0.0)]
    for m in range(1, steps + 1):
        b = loads(mesh, prm, K, m * prm.tau) + history(A, mesh, xs[-1])
        xs.append(solve(A, b, xs[-1]))
    return mesh, A, xs
