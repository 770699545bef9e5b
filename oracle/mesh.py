"""Structured triangulation of the unit square and DoF numbering.

Mesh (Appendix A): ``n`` x ``n`` squares of side ``h = 1/n``, each cut once along the
diagonal from its top-left to its bottom-right corner.  Cell ``(i, j)`` holds

  L(i, j) = {(i, j), (i+1, j), (i, j+1)}      U(i, j) = {(i+1, j+1), (i, j+1), (i+1, j)}

(vertex coordinates in units of h).  Local vertex k of a triangle is opposite its local
edge k:  L: edges (d(i,j), v(i,j), h(i,j));  U: edges (d(i,j), v(i+1,j), h(i,j+1)).

DoFs (Sec. 2.1, Sec. 2.3): P1 displacement (2 per vertex), one face-normal bubble per edge,
one RT0 flux per edge, one P0 pressure per triangle -- 10 DoF types per cell (Sec. 4.2).
The oracle numbers DoFs type by type in the order of ``synthetic.TYPES``; inside a type
row-major over ``[j, i]`` with the shapes of ``synthetic.shapes``.

Pinned by: tests/test_oracle_mesh.py (the triangles tile the square, edge incidence, local
vertex k opposite local edge k, DoF and Dirichlet counts, patch sizes) and, through the
assembled matrices, the App. A stencil pins of tests/test_oracle_assembly.py.
"""
from __future__ import annotations

import numpy as np

import synthetic

TYPES = synthetic.TYPES


class Mesh:
    """DoF numbering of an ``n``-cell grid.

    ``w_essential`` switches the RT0 boundary DoFs from free (natural pressure condition,
    the default reading for the workloads) to constrained (w.n = 0 on the boundary).
    """

    def __init__(self, n: int, w_essential: bool = False):
        assert n >= 1
        self.n = n
        self.w_essential = bool(w_essential)
        self.h = 1.0 / n
        self.shapes = synthetic.shapes(n)
        self.offsets = {}
        off = 0
        for t in TYPES:
            self.offsets[t] = off
            r, c = self.shapes[t]
            off += r * c
        self.ndof = off
        masks = synthetic.dirichlet_masks(n)
        if w_essential:
            masks["wh"][0, :] = masks["wh"][-1, :] = True
            masks["wv"][:, 0] = masks["wv"][:, -1] = True
        self.fixed = self.pack(masks).astype(bool)
        self.free = ~self.fixed
        self.free_idx = np.nonzero(self.free)[0]

    # ----- numbering -------------------------------------------------------------------
    def idx(self, t: str, i, j):
        """Global index of DoF type ``t`` at grid position ``(i, j)`` (arrays allowed)."""
        r, c = self.shapes[t]
        return self.offsets[t] + np.asarray(j) * c + np.asarray(i)

    def pack(self, fields: dict) -> np.ndarray:
        """dict of ``[j, i]`` arrays -> flat vector in the oracle's numbering."""
        return np.concatenate([np.asarray(fields[t], dtype=float).ravel() for t in TYPES])

    def unpack(self, x: np.ndarray) -> dict:
        out = {}
        for t in TYPES:
            r, c = self.shapes[t]
            o = self.offsets[t]
            out[t] = np.array(x[o:o + r * c]).reshape(r, c)
        return out

    # ----- geometry --------------------------------------------------------------------
    def triangles(self):
        """Yield ``(orient, i, j)`` for every triangle, L before U in each cell."""
        for j in range(self.n):
            for i in range(self.n):
                yield "L", i, j
                yield "U", i, j

    @staticmethod
    def tri_vertices(orient: str, i: int, j: int):
        """Vertices (grid units), local vertex k opposite local edge k."""
        if orient == "L":
            return [(i, j), (i + 1, j), (i, j + 1)]
        return [(i + 1, j + 1), (i, j + 1), (i + 1, j)]

    @staticmethod
    def tri_edges(orient: str, i: int, j: int):
        """Edges ``(family, ei, ej)``; local edge k is opposite local vertex k."""
        if orient == "L":
            return [("d", i, j), ("v", i, j), ("h", i, j)]
        return [("d", i, j), ("v", i + 1, j), ("h", i, j + 1)]

    @staticmethod
    def edge_vertices(fam: str, i: int, j: int):
        if fam == "h":
            return (i, j), (i + 1, j)
        if fam == "v":
            return (i, j), (i, j + 1)
        return (i, j + 1), (i + 1, j)

    def tri_dofs(self, orient: str, i, j) -> np.ndarray:
        """The 13 local DoFs of a triangle: ux@v0..v2, uy@v0..v2, bubble@e0..e2,
        RT0@e0..e2, P0.  ``i``, ``j`` may be arrays; the result is then (13, len)."""
        i = np.asarray(i)
        j = np.asarray(j)
        if orient == "L":
            vs = [(i, j), (i + 1, j), (i, j + 1)]
            es = [("d", i, j), ("v", i, j), ("h", i, j)]
        else:
            vs = [(i + 1, j + 1), (i, j + 1), (i + 1, j)]
            es = [("d", i, j), ("v", i + 1, j), ("h", i, j + 1)]
        out = [self.idx("ux", a, b) for a, b in vs]
        out += [self.idx("uy", a, b) for a, b in vs]
        out += [self.idx("b" + f, a, b) for f, a, b in es]
        out += [self.idx("w" + f, a, b) for f, a, b in es]
        out += [self.idx("pL" if orient == "L" else "pU", i, j)]
        return np.array(out, dtype=np.int64)

    def vertex_patch(self, i: int, j: int, with_flow: bool = True) -> list:
        """DoFs of the vertex patch of Fig. 3 (right: 20 DoFs; left, ``with_flow=False``:
        the 8 displacement DoFs), restricted to DoFs that exist and are free.

        Order: ux, uy at the vertex; bubbles on the 6 incident edges; RT0 on those edges;
        P0 on the 6 incident triangles.
        """
        n = self.n
        edges = [("h", i, j), ("v", i, j), ("h", i - 1, j), ("v", i, j - 1),
                 ("d", i - 1, j), ("d", i, j - 1)]
        tris = [("L", i, j), ("L", i - 1, j), ("L", i, j - 1),
                ("U", i - 1, j), ("U", i - 1, j - 1), ("U", i, j - 1)]

        def edge_ok(f, a, b):
            r, c = self.shapes["b" + f]
            return 0 <= a < c and 0 <= b < r

        out = [self.idx("ux", i, j), self.idx("uy", i, j)]
        out += [self.idx("b" + f, a, b) for f, a, b in edges if edge_ok(f, a, b)]
        if with_flow:
            out += [self.idx("w" + f, a, b) for f, a, b in edges if edge_ok(f, a, b)]
            out += [self.idx("pL" if o == "L" else "pU", a, b) for o, a, b in tris
                    if 0 <= a < n and 0 <= b < n]
        out = [int(k) for k in out if self.free[k]]
        return out
