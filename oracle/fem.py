"""Element matrices and global assembly of the reduced-quadrature Biot operator.

Block operator (Sec. 2.3, Eq. block_form_rq; Eq. block_form for the blocks' meaning):

        | A_u^RQ      0          alpha B_u^T |
    A = | 0           tau M_w    tau B_w^T   |
        | alpha B_u   tau B_w    -(1/M) M_p  |

  A_u^RQ  <-  2 mu (eps(u), eps(v)) + lambda (P_Q div u, P_Q div v)      (Sec. 2.3, App. A)
  B_u     <-  -(div u, q)         B_w  <-  -(div w, q)
  M_w     <-  (K^{-1} mu_f w, r)  M_p  <-  (p, q)

Bases (the conventions under which the printed App. A stencils hold):
  * P1 hats for each displacement component;
  * edge bubble  phi_e = 4 lambda_a lambda_b n_e  (a, b the edge's end points), so the bubble
    coefficient is the normal displacement at the edge midpoint;
  * RT0  psi_e  with  psi_e . n_e = 1  on e;
  * P0 indicator of the triangle;
  * global edge normals  n_h = (0, 1),  n_v = (1, 0),  n_d = (1, 1)/sqrt(2).

All integrands are polynomials of degree <= 2 on a triangle, so the three-point
edge-midpoint rule (weights |T|/3) integrates them exactly.  The reduced-quadrature
grad-div term is (1/|T|) (int_T div phi_a)(int_T div phi_b) on each triangle, i.e.
lambda B_u^T M_p^{-1} B_u (App. A).

Pinned by: the interior stencils printed in App. A (tests/test_oracle_assembly.py),
symmetry of A (Sec. 2.1), the local divergence-free functions of Fig. 2, direct-solve
parity on tiny grids and the manufactured-solution convergence rates of Sec. 5.1.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .mesh import Mesh

SQ2 = np.sqrt(2.0)
NORMALS = {"h": np.array([0.0, 1.0]), "v": np.array([1.0, 0.0]), "d": np.array([1.0, 1.0]) / SQ2}


class Params:
    """Physical parameters of one linear solve (one backward-Euler step, Sec. 2.1).

    ``inv_M`` is 1/M (the Biot modulus enters only as 1/M); ``mu_f`` is folded into K.
    ``exact_divdiv`` selects the original discretisation (exact (div u, div v), Sec. 2.1)
    instead of the reduced-quadrature one (Sec. 2.3).
    """

    def __init__(self, lam=1.0, mu=1.0, tau=1.0, alpha=1.0, inv_M=1e-6, exact_divdiv=False):
        self.lam = float(lam)
        self.mu = float(mu)
        self.tau = float(tau)
        self.alpha = float(alpha)
        self.inv_M = float(inv_M)
        self.exact_divdiv = bool(exact_divdiv)

    @staticmethod
    def from_paper(E: float, nu: float, **kw):
        """Lame coefficients from Young's modulus and Poisson ratio (Sec. 2):
        mu = E / (2 + 2 nu),  lambda = E nu / ((1 - 2 nu)(1 + nu))."""
        mu = E / (2.0 + 2.0 * nu)
        lam = E * nu / ((1.0 - 2.0 * nu) * (1.0 + nu))
        return Params(lam=lam, mu=mu, **kw)


# ------------------------------------------------------------------------------------
# Reference quantities on one triangle
# ------------------------------------------------------------------------------------
class Triangle:
    """Geometry and basis functions of one triangle (vertices in physical coordinates)."""

    def __init__(self, X: np.ndarray, edge_fams):
        self.X = np.asarray(X, dtype=float)               # (3, 2)
        M = np.vstack([self.X.T, np.ones(3)])              # lambda = M^{-1} [x, y, 1]
        self.Minv = np.linalg.inv(M)
        self.grad = self.Minv[:, :2]                       # grad lambda_k, rows k
        e1 = self.X[1] - self.X[0]
        e2 = self.X[2] - self.X[0]
        self.area = 0.5 * abs(e1[0] * e2[1] - e1[1] * e2[0])
        self.fams = list(edge_fams)
        self.centroid = self.X.mean(axis=0)
        # local edge k is opposite vertex k: end points (k+1, k+2) mod 3
        self.ends = [((k + 1) % 3, (k + 2) % 3) for k in range(3)]
        self.len = np.array([np.linalg.norm(self.X[b] - self.X[a]) for a, b in self.ends])
        self.nrm = [NORMALS[f] for f in self.fams]
        self.nout = []
        for k, (a, b) in enumerate(self.ends):
            t = self.X[b] - self.X[a]
            nn = np.array([t[1], -t[0]]) / np.linalg.norm(t)
            if np.dot(nn, self.X[a] - self.X[k]) < 0:        # point away from vertex k
                nn = -nn
            self.nout.append(nn)
        # sign s_k = n_e . n_out (+-1)
        self.sgn = np.array([float(np.sign(np.dot(self.nrm[k], self.nout[k]))) for k in range(3)])
        self.mid = np.array([0.5 * (self.X[a] + self.X[b]) for a, b in self.ends])

    def bary(self, x):
        return self.Minv @ np.array([x[0], x[1], 1.0])

    # values and gradients of the 9 displacement basis functions at a point ----------
    def u_basis(self, x):
        """Returns (values (9, 2), gradients (9, 2, 2) with G[c, s] = d u_c / d x_s)."""
        lam = self.bary(x)
        vals = np.zeros((9, 2))
        grads = np.zeros((9, 2, 2))
        for k in range(3):                      # ux, uy hats
            vals[k, 0] = lam[k]
            grads[k, 0, :] = self.grad[k]
            vals[3 + k, 1] = lam[k]
            grads[3 + k, 1, :] = self.grad[k]
        for k, (a, b) in enumerate(self.ends):  # bubbles 4 la lb n_e
            ne = self.nrm[k]
            vals[6 + k] = 4.0 * lam[a] * lam[b] * ne
            g = 4.0 * (lam[a] * self.grad[b] + lam[b] * self.grad[a])
            grads[6 + k] = np.outer(ne, g)
        return vals, grads

    def w_basis(self, x):
        """RT0 values (3, 2) with psi_k . n_k = 1 on edge k, and divergences (3,)."""
        vals = np.zeros((3, 2))
        divs = np.zeros(3)
        for k in range(3):
            c = self.sgn[k] * self.len[k] / (2.0 * self.area)
            vals[k] = c * (np.asarray(x) - self.X[k])
            divs[k] = 2.0 * c
        return vals, divs

    def quad(self):
        """Edge-midpoint rule: points and weights (exact up to degree 2)."""
        return self.mid, np.full(3, self.area / 3.0)


def element_parts(tri: Triangle):
    """Unit-parameter element integrals on one triangle.

    Returns dict with
      Aeps (9, 9)  int eps(phi_a):eps(phi_b)
      Ddiv (9, 9)  int div phi_a div phi_b   (exact: the divergence of a bubble is linear)
      g    (9,)    int div phi_a
      Mw   (3, 3)  int psi_a . psi_b
      dw   (3,)    int div psi_a
      area
    """
    pts, wts = tri.quad()
    Aeps = np.zeros((9, 9))
    Ddiv = np.zeros((9, 9))
    g = np.zeros(9)
    Mw = np.zeros((3, 3))
    dw = np.zeros(3)
    for x, wq in zip(pts, wts):
        _, G = tri.u_basis(x)
        eps = 0.5 * (G + np.transpose(G, (0, 2, 1)))
        Aeps += wq * np.einsum("aij,bij->ab", eps, eps)
        dv = np.trace(G, axis1=1, axis2=2)
        Ddiv += wq * np.outer(dv, dv)
        g += wq * dv
        psi, divs = tri.w_basis(x)
        Mw += wq * psi @ psi.T
        dw += wq * divs
    return {"Aeps": Aeps, "Ddiv": Ddiv, "g": g, "Mw": Mw, "dw": dw, "area": tri.area}


def element_matrix(parts: dict, prm: Params, kinv: float) -> np.ndarray:
    """13 x 13 element matrix of the reduced-quadrature operator (Sec. 2.3) in local
    order (ux0..2, uy0..2, b0..2, w0..2, p).  With ``prm.exact_divdiv`` the grad-div term is
    lambda (div u, div v) integrated exactly: the original discretisation of Eq. block_form
    (Sec. 2.1), which Sec. 2.2 and Table 1 show is not solver-friendly."""
    E = np.zeros((13, 13))
    g = parts["g"]
    if getattr(prm, "exact_divdiv", False):
        E[:9, :9] = 2.0 * prm.mu * parts["Aeps"] + prm.lam * parts["Ddiv"]
    else:
        E[:9, :9] = 2.0 * prm.mu * parts["Aeps"] + prm.lam * np.outer(g, g) / parts["area"]
    E[:9, 12] = E[12, :9] = -prm.alpha * g                         # alpha B_u,  B_u = -(div u, q)
    E[9:12, 9:12] = prm.tau * kinv * parts["Mw"]                    # tau M_w
    E[9:12, 12] = E[12, 9:12] = -prm.tau * parts["dw"]              # tau B_w,  B_w = -(div w, q)
    E[12, 12] = -prm.inv_M * parts["area"]                          # -(1/M) M_p
    return E


def reference_triangles(n: float):
    """The two triangle shapes of the mesh (L and U of cell (0, 0)); spacing h = 1/n."""
    h = 1.0 / n
    out = {}
    for o in ("L", "U"):
        X = np.array(Mesh.tri_vertices(o, 0, 0), dtype=float) * h
        out[o] = Triangle(X, [e[0] for e in Mesh.tri_edges(o, 0, 0)])
    return out


def assemble(mesh: Mesh, prm: Params, kinv_L: np.ndarray, kinv_U: np.ndarray,
             h: float = None) -> sp.csr_matrix:
    """Global operator on all DoFs, constrained rows and columns removed (zeroed).

    ``kinv_L``, ``kinv_U``: per-triangle K^{-1} arrays ``(n, n)`` indexed ``[j, i]``.
    Triangles of equal shape share all element integrals; only the RT0 mass is scaled by
    the triangle's K^{-1}.  Element loop vectorised over triangles of one shape.
    ``h`` (default 1/n) overrides the cell size: the local Fourier analysis reads the
    interior stencils of a grid with spacing h from a small patch of cells.
    """
    n = mesh.n
    tris = reference_triangles(n if h is None else 1.0 / h)
    rows, cols, vals = [], [], []
    jj, ii = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    for o in ("L", "U"):
        parts = element_parts(tris[o])
        kin = (kinv_L if o == "L" else kinv_U).ravel()
        E0 = element_matrix(parts, prm, 0.0)                 # everything except the RT0 mass
        Mw = prm.tau * parts["Mw"]
        dofs = mesh.tri_dofs(o, ii.ravel(), jj.ravel()).T            # (n*n, 13)
        V = np.broadcast_to(E0, (n * n, 13, 13)).copy()
        V[:, 9:12, 9:12] += kin[:, None, None] * Mw[None]
        rows.append(np.repeat(dofs, 13, axis=1).ravel())
        cols.append(np.tile(dofs, (1, 13)).ravel())
        vals.append(V.ravel())
    rows = np.concatenate(rows)
    cols = np.concatenate(cols)
    vals = np.concatenate(vals)
    A = sp.coo_matrix((vals, (rows, cols)), shape=(mesh.ndof, mesh.ndof)).tocsr()
    A.sum_duplicates()
    keep = sp.diags(mesh.free.astype(float))
    A = (keep @ A @ keep).tocsr()
    A.eliminate_zeros()
    return A


def kinv_from_k(K_L, K_U):
    return 1.0 / np.asarray(K_L, dtype=float), 1.0 / np.asarray(K_U, dtype=float)


def apply(A: sp.csr_matrix, x: np.ndarray) -> np.ndarray:
    """y = A x (FP64 sparse matrix-vector product)."""
    return A @ x


def residual(A: sp.csr_matrix, b: np.ndarray, x: np.ndarray) -> np.ndarray:
    """r = b - A x."""
    return b - A @ x


def block(A, mesh: Mesh, rtypes, ctypes_):
    """Sub-block of A with rows of the DoF types ``rtypes`` and columns ``ctypes_``."""
    def sel(ts):
        return np.concatenate([np.arange(mesh.offsets[t], mesh.offsets[t] + np.prod(mesh.shapes[t]))
                               for t in ts])
    return A[sel(rtypes)][:, sel(ctypes_)], sel(rtypes), sel(ctypes_)


U_TYPES = ("ux", "uy", "bh", "bv", "bd")
W_TYPES = ("wh", "wv", "wd")
P_TYPES = ("pL", "pU")


def type_mask(mesh: Mesh, ts) -> np.ndarray:
    m = np.zeros(mesh.ndof, dtype=bool)
    for t in ts:
        o = mesh.offsets[t]
        m[o:o + int(np.prod(mesh.shapes[t]))] = True
    return m


def apply_rows(mesh: Mesh, prm: Params, kinv_L: np.ndarray, kinv_U: np.ndarray, x: np.ndarray,
               rows) -> np.ndarray:
    """(A x)[rows] computed one row at a time by summing the element contributions of the
    triangles that hold each row's DoF (for sampled checks on grids too large to assemble).
    Constrained rows return 0 and constrained entries of x are ignored.

    Pinned by: equality with the assembled operator on every row of an 8-cell grid
    (lognormal K, three parameter sets; tests/test_oracle_assembly.py)."""
    n = mesh.n
    tris = reference_triangles(n)
    parts = {o: element_parts(tris[o]) for o in ("L", "U")}
    base = {o: element_matrix(parts[o], prm, 0.0) for o in ("L", "U")}
    xf = np.where(mesh.free, x, 0.0)
    out = np.zeros(len(rows))
    for k, r in enumerate(rows):
        if not mesh.free[r]:
            continue
        t = None
        for tt in TYPES_ALL:
            o_ = mesh.offsets[tt]
            rr, cc = mesh.shapes[tt]
            if o_ <= r < o_ + rr * cc:
                t = tt
                j, i = divmod(r - o_, cc)
        acc = 0.0
        for cj in range(max(0, j - 1), min(n, j + 1)):
            for ci in range(max(0, i - 1), min(n, i + 1)):
                for o in ("L", "U"):
                    dofs = mesh.tri_dofs(o, ci, cj)
                    hit = np.nonzero(dofs == r)[0]
                    if hit.size == 0:
                        continue
                    E = base[o].copy()
                    kin = (kinv_L if o == "L" else kinv_U)[cj, ci]
                    E[9:12, 9:12] += prm.tau * kin * parts[o]["Mw"]
                    acc += float(E[hit[0]] @ xf[dofs])
        out[k] = acc
    return out


TYPES_ALL = ("ux", "uy", "bh", "bv", "bd", "wh", "wv", "wd", "pL", "pU")
