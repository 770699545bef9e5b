"""Adjoint gradients of a loss on the pressure with respect to the per-triangle
log-permeability theta_T = log K_T and the Lame coefficients (CPU oracle, FP64).

For A(theta, lambda, mu) x = b and a loss L(p(x)):
    A^T xi = dL/dx  (A is symmetric by the scaling of Sec. 2.1, so A xi = dL/dx),
    dL/dq = -xi^T (dA/dq) x   for every parameter q.
With the element matrices of Sec. 2.3 (see fem.py):
    dA/dtheta_T = -e^{-theta_T} tau M_T        (the RT0 mass of triangle T at unit K)
    dA/dlambda  = sum_T g_T g_T^T / |T|         (reduced-quadrature grad-div, u-block)
    dA/dmu      = sum_T 2 A_eps,T               (u-block)
so  dL/dtheta_T = e^{-theta_T} xi_w,T^T (tau M_T) w_T,
    dL/dlambda  = -sum_T (g_T . xi_u,T)(g_T . u_T) / |T|,
    dL/dmu      = -sum_T xi_u,T^T (2 A_eps,T) u_T.

Pinned by central finite differences of J(theta) = ||p - p_obs||^2 computed with direct
solves (tests/test_oracle_adjoint.py).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse.linalg as spla

from . import fem
from .mesh import Mesh


def direct_solve(A, mesh: Mesh, b: np.ndarray) -> np.ndarray:
    fi = mesh.free_idx
    x = np.zeros_like(b)
    x[fi] = spla.spsolve(A[fi][:, fi].tocsc(), b[fi])
    return x


def pressure(mesh: Mesh, x: np.ndarray) -> np.ndarray:
    """P0 coefficients as an array (2, n, n): [0] lower-left, [1] upper-right triangles."""
    f = mesh.unpack(x)
    return np.stack([f["pL"], f["pU"]])


def embed_pressure(mesh: Mesh, gp: np.ndarray) -> np.ndarray:
    """A vector that is gp (2, n, n) on the P0 DoFs and zero elsewhere."""
    f = {t: np.zeros(s) for t, s in mesh.shapes.items()}
    f["pL"] = gp[0]
    f["pU"] = gp[1]
    return mesh.pack(f)


def gradients(mesh: Mesh, prm: fem.Params, theta_L, theta_U, x: np.ndarray, xi: np.ndarray):
    """(dL/dtheta as (2, n, n), dL/dlambda, dL/dmu) from the forward solution x and the
    adjoint solution xi (element loop, vectorised over the triangles of one shape)."""
    n = mesh.n
    tris = fem.reference_triangles(n)
    jj, ii = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    dth = np.zeros((2, n, n))
    dlam = 0.0
    dmu = 0.0
    xf = np.where(mesh.free, x, 0.0)
    xif = np.where(mesh.free, xi, 0.0)
    for k, o in enumerate(("L", "U")):
        parts = fem.element_parts(tris[o])
        dofs = mesh.tri_dofs(o, ii.ravel(), jj.ravel()).T           # (n*n, 13)
        xl = xf[dofs]
        yl = xif[dofs]
        theta = (theta_L if o == "L" else theta_U).ravel()
        Mt = prm.tau * parts["Mw"]
        dth[k] = (np.exp(-theta) * np.einsum("ta,ab,tb->t", yl[:, 9:12], Mt, xl[:, 9:12])).reshape(n, n)
        g = parts["g"]
        dlam -= float(np.sum((yl[:, :9] @ g) * (xl[:, :9] @ g)) / parts["area"])
        dmu -= float(np.einsum("ta,ab,tb->", yl[:, :9], 2.0 * parts["Aeps"], xl[:, :9]))
    return dth, dlam, dmu


def misfit_gradients(n: int, prm: fem.Params, theta_L, theta_U, b: np.ndarray, p_obs: np.ndarray):
    """J = ||p - p_obs||^2 and its gradients by one forward and one adjoint direct solve."""
    mesh = Mesh(n)
    A = fem.assemble(mesh, prm, np.exp(-theta_L), np.exp(-theta_U))
    x = direct_solve(A, mesh, b)
    r = pressure(mesh, x) - p_obs
    J = float(np.sum(r * r))
    xi = direct_solve(A, mesh, embed_pressure(mesh, 2.0 * r))
    dth, dlam, dmu = gradients(mesh, prm, theta_L, theta_U, x, xi)
    return J, dth, dlam, dmu, x, xi


def misfit(n: int, prm: fem.Params, theta_L, theta_U, b: np.ndarray, p_obs: np.ndarray) -> float:
    mesh = Mesh(n)
    A = fem.assemble(mesh, prm, np.exp(-theta_L), np.exp(-theta_U))
    x = direct_solve(A, mesh, b)
    r = pressure(mesh, x) - p_obs
    return float(np.sum(r * r))
