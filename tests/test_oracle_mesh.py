"""Pins of the oracle's structured triangulation and DoF numbering (oracle/mesh.py; App. A's
mesh, the spaces of Sec. 2.1 / 2.3, the vertex patches of Fig. 3), against geometry and
counting rather than against the module's own tables:

* the 2n^2 triangles tile the unit square (positive orientation, areas summing to 1),
  every interior edge borders exactly two triangles and every boundary edge one;
* local vertex k of a triangle is the vertex not on its local edge k;
* DoF counts: 2(n+1)^2 displacement + (3n^2 + 2n) bubble + (3n^2 + 2n) flux + 2n^2 pressure;
  the Dirichlet displacement condition fixes ux, uy on the 4n boundary vertices and the
  bubbles on the 4n boundary edges (2,498 free DoFs at n = 16);
* a triangle's 13 DoF indices are distinct and every DoF belongs to some triangle;
* an interior vertex patch has 20 DoFs, 2 + 6 + 6 + 6."""
from collections import Counter

import numpy as np
import pytest

from oracle.mesh import Mesh


@pytest.mark.parametrize("n", [1, 2, 5, 8])
def test_triangles_tile_the_square(n):
    m = Mesh(n)
    area = 0.0
    edge_use = Counter()
    for o, i, j in m.triangles():
        V = np.array(Mesh.tri_vertices(o, i, j), float) / n
        a = 0.5 * ((V[1, 0] - V[0, 0]) * (V[2, 1] - V[0, 1]) - (V[2, 0] - V[0, 0]) * (V[1, 1] - V[0, 1]))
        assert a > 0                                    # counter-clockwise
        area += a
        verts = Mesh.tri_vertices(o, i, j)
        for k, (f, ei, ej) in enumerate(Mesh.tri_edges(o, i, j)):
            ev = set(Mesh.edge_vertices(f, ei, ej))
            assert ev == set(verts) - {verts[k]}        # local edge k is opposite vertex k
            edge_use[(f, ei, ej)] += 1
    assert abs(area - 1.0) < 1e-14
    for (f, ei, ej), c in edge_use.items():
        a, b = Mesh.edge_vertices(f, ei, ej)
        on_boundary = (a[0] == b[0] and a[0] in (0, n)) or (a[1] == b[1] and a[1] in (0, n))
        assert c == (1 if on_boundary else 2), (f, ei, ej, c)
    assert len(edge_use) == 3 * n * n + 2 * n


@pytest.mark.parametrize("n", [1, 3, 16])
def test_dof_counts(n):
    m = Mesh(n)
    assert m.ndof == 2 * (n + 1) ** 2 + 2 * (3 * n * n + 2 * n) + 2 * n * n
    # fixed: ux, uy on the 4n boundary vertices, bubbles on the 4n boundary edges
    assert int(m.fixed.sum()) == 2 * 4 * n + 4 * n
    if n == 16:
        assert int(m.free.sum()) == 2498


def test_triangle_dofs_cover_every_dof_once_per_use():
    n = 4
    m = Mesh(n)
    seen = np.zeros(m.ndof, int)
    for o, i, j in m.triangles():
        d = m.tri_dofs(o, i, j)
        assert len(set(d.tolist())) == 13
        seen[d] += 1
    assert np.all(seen > 0)
    # pressures belong to one triangle, vertex DoFs to up to six
    assert seen[m.idx("pL", np.arange(n), 0)].max() == 1
    assert seen[m.idx("ux", 2, 2)] == 6 and seen[m.idx("ux", 0, 0)] == 1


def test_interior_vertex_patch_has_twenty_dofs():
    m = Mesh(8)
    p = m.vertex_patch(3, 4)
    assert len(p) == 20 and len(set(p)) == 20
    assert len(m.vertex_patch(3, 4, with_flow=False)) == 8
