"""Grid transfers between an ``N``-cell grid and the ``2N``-cell grid (Sec. 3, Sec. 3.1).

Block interpolation P = diag(P_u, P_w, P_p) (Eq. block_interp) and R = P^T:

  * P_p: canonical P0 interpolation (each fine triangle takes its parent's value).
  * P_w: canonical RT0 interpolation: the fine DoF is the normal component (w.r.t. the
    fine edge's global normal) of the coarse RT0 field at the fine edge midpoint.
  * P_u: divergence-preserving interpolation (Sec. 3.1).  First the canonical finite-element
    interpolant of the coarse P1+bubble function: fine P1 DoFs are point values at fine
    vertices; the fine bubble DoF of an edge is the normal component, at the midpoint, of the
    function minus its P1 interpolant (the bubble coefficient under the basis
    4 lambda_a lambda_b n_e).  Then, for each of the three corner children t of a coarse
    triangle (Fig. 4), the bubble DoF on t's interior edge is overwritten so that the net
    flux of the fine function through the boundary of t vanishes (Eq. divfreefine); the
    flux of P1 + bubble data through an edge e is |e| (u(a)+u(b))/2 . n_out +
    (2/3)|e| c_e (n_e . n_out).

The construction runs coarse triangle by coarse triangle; a fine DoF on a coarse edge gets
the same value from either neighbour, so values are set, not summed.

Pinned by: the App. B restriction-symbol coefficients (1/4, sqrt2/8, 5 sqrt2/8, -1,
3 sqrt2/16, 3/8, the 7-point P1 weights), zero flux of every P_u column on corner triangles,
the identity B_u,h P_u = Q B_u,H (divergence only in the interior child), and the nested-space
Galerkin identities P_w^T M_w P_w = M_w,H, P_p^T B_w P_w = B_w,H, P_p^T M_p P_p = M_p,H
(tests/test_oracle_transfer.py).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .fem import Triangle
from .mesh import Mesh


def fine_edge(p, q):
    """Structured edge ``(family, i, j)`` through two adjacent vertices of one grid."""
    (i0, j0), (i1, j1) = p, q
    if j0 == j1:
        return "h", min(i0, i1), j0
    if i0 == i1:
        return "v", i0, min(j0, j1)
    assert abs(i0 - i1) == 1 and abs(j0 - j1) == 1 and (i1 - i0) * (j1 - j0) < 0
    return "d", min(i0, i1), min(j0, j1)


def fine_triangle(verts):
    """``(orient, i, j)`` of the structured triangle with the given vertex set."""
    imin = min(v[0] for v in verts)
    jmin = min(v[1] for v in verts)
    return ("L" if (imin, jmin) in verts else "U"), imin, jmin


def _tri_object(verts, h):
    """Triangle with local vertex k opposite local edge k, from grid vertices."""
    X = np.array(verts, dtype=float) * h
    fams = [fine_edge(verts[(k + 1) % 3], verts[(k + 2) % 3])[0] for k in range(3)]
    return Triangle(X, fams)


_CACHE = {}


def prolongation(fine: Mesh, coarse: Mesh) -> sp.csr_matrix:
    """P: coarse vector -> fine vector, rows/columns of constrained DoFs removed (zeroed).
    P depends only on the grids, so it is built once per grid pair and reused."""
    key = (fine.n, coarse.n, fine.w_essential, coarse.w_essential)
    if key not in _CACHE:
        _CACHE[key] = _prolongation(fine, coarse)
    return _CACHE[key].copy()


def _prolongation(fine: Mesh, coarse: Mesh) -> sp.csr_matrix:
    assert fine.n == 2 * coarse.n
    h = fine.h
    H = coarse.h
    entries = {}

    def put(r, c, v):
        if v != 0.0:
            entries[(int(r), int(c))] = float(v)

    for o, I, J in coarse.triangles():
        cv = Mesh.tri_vertices(o, I, J)                     # coarse grid units
        tc = _tri_object(cv, H)
        cdofs = coarse.tri_dofs(o, I, J)                   # 13 coarse DoFs
        A = [(2 * a, 2 * b) for a, b in cv]                # coarse vertices in fine units
        Mid = [((A[(k + 1) % 3][0] + A[(k + 2) % 3][0]) // 2,
                (A[(k + 1) % 3][1] + A[(k + 2) % 3][1]) // 2) for k in range(3)]
        fverts = A + Mid
        # edges: 6 halves of coarse edges, 3 interior edges (of the interior child)
        halves = []
        for k in range(3):
            a, b = A[(k + 1) % 3], A[(k + 2) % 3]
            halves += [(a, Mid[k]), (Mid[k], b)]
        interior = [(Mid[1], Mid[2]), (Mid[2], Mid[0]), (Mid[0], Mid[1])]
        children = [[A[0], Mid[2], Mid[1]], [A[1], Mid[0], Mid[2]], [A[2], Mid[1], Mid[0]]]
        inner_child = [Mid[0], Mid[1], Mid[2]]

        # ---- P_u: canonical interpolation of the 9 coarse displacement basis functions
        for a in range(9):
            col = cdofs[a]

            def f(p):
                vals, _ = tc.u_basis(np.array(p, dtype=float) * h)
                return vals[a]

            fv = {p: f(p) for p in fverts}
            for p in fverts:
                put(fine.idx("ux", *p), col, fv[p][0])
                put(fine.idx("uy", *p), col, fv[p][1])
            bub = {}
            for (p, q) in halves:
                fam, i, j = fine_edge(p, q)
                mid = (np.array(p, float) + np.array(q, float)) * 0.5
                nvec = {"h": np.array([0.0, 1.0]), "v": np.array([1.0, 0.0]),
                        "d": np.array([1.0, 1.0]) / np.sqrt(2.0)}[fam]
                vm, _ = tc.u_basis(mid * h)
                c = float(np.dot(nvec, vm[a] - 0.5 * (fv[p] + fv[q])))
                bub[frozenset((p, q))] = c
                put(fine.idx("b" + fam, i, j), col, c)
            # ---- divergence fix on the three corner children
            for verts in children:
                t = _tri_object(verts, h)
                flux = 0.0
                kint = None
                for k in range(3):
                    pa, pb = verts[(k + 1) % 3], verts[(k + 2) % 3]
                    key = frozenset((pa, pb))
                    flux += t.len[k] * 0.5 * float(np.dot(fv[pa] + fv[pb], t.nout[k]))
                    if key in bub:
                        flux += (2.0 / 3.0) * t.len[k] * bub[key] * t.sgn[k]
                    else:
                        kint = k
                pa, pb = verts[(kint + 1) % 3], verts[(kint + 2) % 3]
                fam, i, j = fine_edge(pa, pb)
                c = -flux / ((2.0 / 3.0) * t.len[kint] * t.sgn[kint])
                put(fine.idx("b" + fam, i, j), col, c)

        # ---- P_w: canonical RT0 interpolation of the 3 coarse flux basis functions
        for a in range(3):
            col = cdofs[9 + a]
            for (p, q) in halves + interior:
                fam, i, j = fine_edge(p, q)
                mid = (np.array(p, float) + np.array(q, float)) * 0.5 * h
                psi, _ = tc.w_basis(mid)
                nvec = {"h": np.array([0.0, 1.0]), "v": np.array([1.0, 0.0]),
                        "d": np.array([1.0, 1.0]) / np.sqrt(2.0)}[fam]
                put(fine.idx("w" + fam, i, j), col, float(np.dot(psi[a], nvec)))

        # ---- P_p: injection into the four children
        for verts in children + [inner_child]:
            fo, fi, fj = fine_triangle(verts)
            put(fine.idx("pL" if fo == "L" else "pU", fi, fj), cdofs[12], 1.0)

    r = np.array([k[0] for k in entries], dtype=np.int64)
    c = np.array([k[1] for k in entries], dtype=np.int64)
    v = np.array(list(entries.values()))
    P = sp.coo_matrix((v, (r, c)), shape=(fine.ndof, coarse.ndof)).tocsr()
    P = (sp.diags(fine.free.astype(float)) @ P @ sp.diags(coarse.free.astype(float))).tocsr()
    P.eliminate_zeros()
    return P


def restriction(P: sp.csr_matrix) -> sp.csr_matrix:
    """R = P^T (Sec. 3)."""
    return P.T.tocsr()
