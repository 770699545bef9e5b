"""Pins of the oracle's assembly against what the paper prints (CPU only).

* App. A interior stencils of 2 mu A_eps (P1-P1, P1x-P1y, bubble-bubble, P1-bubble), M_w,
  M_p, B_u and B_w (the symbols of App. A written out as stencil entries);
* symmetry of the block operator (Sec. 2.1: the scaling makes the system symmetric);
* the local divergence-free space around a vertex under reduced quadrature (Sec. 2.3,
  Fig. 2): dimension 3, and the pure-bubble member has Fig. 2's rotational sign pattern;
* the exact solution of a tiny system against a dense LU (numpy).
"""
import numpy as np
import pytest

import synthetic
from oracle import fem
from oracle.mesh import Mesh

S2 = np.sqrt(2.0)


def build(n=8, lam=1.0, mu=1.0, tau=1.0, alpha=1.0, inv_M=1.0, k=1.0):
    m = Mesh(n)
    prm = fem.Params(lam=lam, mu=mu, tau=tau, alpha=alpha, inv_M=inv_M)
    kinv = np.full((n, n), 1.0 / k)
    return m, prm, fem.assemble(m, prm, kinv, kinv)


def entry(A, m, ta, ia, ja, tb, ib, jb):
    return A[m.idx(ta, ia, ja), m.idx(tb, ib, jb)]


@pytest.fixture(scope="module")
def elastic():
    """2 mu A_eps alone: lambda = 0, alpha = 0 (mu = 1.7 to catch a dropped factor)."""
    return build(n=8, lam=0.0, mu=1.7, alpha=0.0)


def test_p1_p1_stencil(elastic):
    # App. A: P1 x-component stencil [[., -mu, .], [-2mu, 6mu, -2mu], [., -mu, .]]
    m, prm, A = elastic
    mu, i, j = prm.mu, 4, 4
    assert entry(A, m, "ux", i, j, "ux", i, j) == pytest.approx(6 * mu, rel=1e-14)
    assert entry(A, m, "ux", i, j, "ux", i + 1, j) == pytest.approx(-2 * mu, rel=1e-14)
    assert entry(A, m, "ux", i, j, "ux", i - 1, j) == pytest.approx(-2 * mu, rel=1e-14)
    assert entry(A, m, "ux", i, j, "ux", i, j + 1) == pytest.approx(-mu, rel=1e-14)
    assert entry(A, m, "ux", i, j, "ux", i, j - 1) == pytest.approx(-mu, rel=1e-14)
    assert abs(entry(A, m, "ux", i, j, "ux", i + 1, j - 1)) < 1e-14
    # y-component: the 90 degree rotation
    assert entry(A, m, "uy", i, j, "uy", i, j + 1) == pytest.approx(-2 * mu, rel=1e-14)
    assert entry(A, m, "uy", i, j, "uy", i + 1, j) == pytest.approx(-mu, rel=1e-14)


def test_p1x_p1y_stencil(elastic):
    # App. A: [[mu/2, -mu/2, .], [-mu/2, mu, -mu/2], [., -mu/2, mu/2]]  (rows: y = +1, 0, -1)
    m, prm, A = elastic
    mu, i, j = prm.mu, 4, 4
    want = {(-1, 1): mu / 2, (0, 1): -mu / 2, (-1, 0): -mu / 2, (0, 0): mu, (1, 0): -mu / 2,
            (0, -1): -mu / 2, (1, -1): mu / 2, (1, 1): 0.0, (-1, -1): 0.0}
    for (di, dj), v in want.items():
        assert entry(A, m, "ux", i, j, "uy", i + di, j + dj) == pytest.approx(v, abs=1e-14)


def test_bubble_bubble_stencil(elastic):
    # App. A bubble symbol mu [[28/3, -(10 sqrt2/3) cos(t1/2), -(10 sqrt2/3) cos(t2/2)],
    # [., 8, (4/3) cos((t1-t2)/2)], [., ., 8]]: diagonals 28mu/3 and 8mu, d-edge to each of
    # its two adjacent axis edges of a family -5 sqrt2 mu/3, h-v pairs of a triangle 2mu/3.
    m, prm, A = elastic
    mu, i, j = prm.mu, 3, 4
    assert entry(A, m, "bd", i, j, "bd", i, j) == pytest.approx(28 * mu / 3, rel=1e-14)
    assert entry(A, m, "bh", i, j, "bh", i, j) == pytest.approx(8 * mu, rel=1e-14)
    assert entry(A, m, "bv", i, j, "bv", i, j) == pytest.approx(8 * mu, rel=1e-14)
    # d(i,j) shares a triangle with v(i,j) (L) and v(i+1,j) (U)
    assert entry(A, m, "bd", i, j, "bv", i, j) == pytest.approx(-5 * S2 * mu / 3, rel=1e-14)
    assert entry(A, m, "bd", i, j, "bv", i + 1, j) == pytest.approx(-5 * S2 * mu / 3, rel=1e-14)
    assert entry(A, m, "bd", i, j, "bh", i, j) == pytest.approx(-5 * S2 * mu / 3, rel=1e-14)
    assert entry(A, m, "bd", i, j, "bh", i, j + 1) == pytest.approx(-5 * S2 * mu / 3, rel=1e-14)
    # h(i,j) and v(i,j) share L(i,j); h(i,j+1) and v(i+1,j) share U(i,j)
    assert entry(A, m, "bh", i, j, "bv", i, j) == pytest.approx(2 * mu / 3, rel=1e-14)
    assert entry(A, m, "bh", i, j + 1, "bv", i + 1, j) == pytest.approx(2 * mu / 3, rel=1e-14)


def test_p1_bubble_stencil(elastic):
    # App. A P1-to-bubble symbol (8mu/3)[sqrt2 (cos((t1-t2)/2) - cos((t1+t2)/2)), ...]:
    # entries +-(4 sqrt2/3) mu to d-bubbles, +-(4/3) mu to the axis bubbles of one family.
    m, prm, A = elastic
    mu, i, j = prm.mu, 4, 4
    row = A[m.idx("ux", i, j)].toarray().ravel()
    vals = []
    for t in ("bd", "bh", "bv"):
        o = m.offsets[t]
        seg = row[o:o + int(np.prod(m.shapes[t]))]
        vals.append(sorted(np.round(seg[np.abs(seg) > 1e-13] / mu, 12)))
    c = round(4 * S2 / 3, 12)
    assert vals[0] == [-c, -c, c, c]
    assert vals[1] == []                     # ux does not couple to h-edge (normal (0,1)) bubbles
    assert vals[2] == [-4 / 3, -4 / 3, 4 / 3, 4 / 3] or np.allclose(vals[2], [-4 / 3, -4 / 3, 4 / 3, 4 / 3])


def test_darcy_and_pressure_mass():
    # App. A: M_w = (mu_f h^2 / 3k)[[2,0,0],[0,2,-cos((t1-t2)/2)],[0,-cos,2]], M_p = (h^2/2) I
    n, k, tau, invM = 8, 0.37, 1.0, 2.0
    m, prm, A = build(n=n, k=k, tau=tau, inv_M=invM)
    h = 1.0 / n
    i, j = 3, 4
    for t in ("wh", "wv", "wd"):
        assert entry(A, m, t, i, j, t, i, j) == pytest.approx(2 * h * h / (3 * k), rel=1e-13)
    assert entry(A, m, "wh", i, j, "wv", i, j) == pytest.approx(-h * h / (6 * k), rel=1e-13)
    assert abs(entry(A, m, "wd", i, j, "wh", i, j)) < 1e-15
    assert abs(entry(A, m, "wd", i, j, "wv", i, j)) < 1e-15
    assert entry(A, m, "pL", i, j, "pL", i, j) == pytest.approx(-invM * h * h / 2, rel=1e-13)


def test_divergence_blocks():
    # App. A: B_u symbol h[-2sqrt2/3, (2/3)e^{-it1/2}, (2/3)e^{-it2/2}, -(1/2)(e^{it1/2}-e^{-it1/2})e^{-it2/2}, ...]
    # and B_w symbol h[[-sqrt2, e^{-it1/2}, e^{-it2/2}], [sqrt2, -e^{it1/2}, -e^{it2/2}]]
    n, alpha, tau = 8, 1.3, 0.7
    m, prm, A = build(n=n, alpha=alpha, tau=tau)
    h = 1.0 / n
    i, j = 3, 4
    assert entry(A, m, "pL", i, j, "bd", i, j) == pytest.approx(-alpha * 2 * S2 / 3 * h, rel=1e-13)
    assert entry(A, m, "pL", i, j, "bv", i, j) == pytest.approx(alpha * 2 / 3 * h, rel=1e-13)
    assert entry(A, m, "pL", i, j, "bh", i, j) == pytest.approx(alpha * 2 / 3 * h, rel=1e-13)
    assert entry(A, m, "pL", i, j, "ux", i + 1, j) == pytest.approx(-alpha * h / 2, rel=1e-13)
    assert entry(A, m, "pL", i, j, "ux", i, j) == pytest.approx(alpha * h / 2, rel=1e-13)
    assert entry(A, m, "pU", i, j, "bd", i, j) == pytest.approx(alpha * 2 * S2 / 3 * h, rel=1e-13)
    assert entry(A, m, "pL", i, j, "wd", i, j) == pytest.approx(-tau * S2 * h, rel=1e-13)
    assert entry(A, m, "pL", i, j, "wv", i, j) == pytest.approx(tau * h, rel=1e-13)
    assert entry(A, m, "pL", i, j, "wh", i, j) == pytest.approx(tau * h, rel=1e-13)
    assert entry(A, m, "pU", i, j, "wd", i, j) == pytest.approx(tau * S2 * h, rel=1e-13)
    assert entry(A, m, "pU", i, j, "wv", i + 1, j) == pytest.approx(-tau * h, rel=1e-13)
    assert entry(A, m, "pU", i, j, "wh", i, j + 1) == pytest.approx(-tau * h, rel=1e-13)


def test_grad_div_is_reduced_quadrature():
    # A_u^RQ = 2 mu A_eps + lambda B_u^T M_p^{-1} B_u  (App. A)
    n = 6
    m, prm, A = build(n=n, lam=3.3, mu=0.9, alpha=0.0)
    _, _, A0 = build(n=n, lam=0.0, mu=0.9, alpha=0.0)
    _, _, Ab = build(n=n, lam=1.0, mu=0.0, alpha=1.0, inv_M=1.0)
    u = fem.type_mask(m, fem.U_TYPES) & m.free
    p = fem.type_mask(m, fem.P_TYPES)
    Bu = Ab[p][:, u].toarray()                          # alpha B_u with alpha = 1
    Mp = -Ab[p][:, p].diagonal()                        # (1/M) M_p with 1/M = 1
    want = A0[u][:, u].toarray() + 3.3 * Bu.T @ np.diag(1.0 / Mp) @ Bu
    assert np.allclose(A[u][:, u].toarray(), want, rtol=1e-12, atol=1e-12)


def test_symmetric():
    m, prm, A = build(n=7, lam=12.0, mu=0.4, tau=0.3, alpha=0.8, inv_M=0.01)
    assert abs(A - A.T).max() < 1e-13 * abs(A).max()


def test_local_divergence_free_space():
    # Sec. 2.3 / Fig. 2: three divergence-free functions supported around each vertex
    n, i, j = 6, 3, 3
    m, prm, A = build(n=n, alpha=1.0)
    patch = m.vertex_patch(i, j, with_flow=False)            # ux, uy, 6 bubbles
    p = np.nonzero(fem.type_mask(m, fem.P_TYPES))[0]
    B = A[p][:, patch].toarray()
    s = np.linalg.svd(B, compute_uv=False)
    assert np.sum(s > 1e-12 * s[0]) == 5                      # 8 - 3
    # the pure-bubble member: signs of Fig. 2 (left) on (h(i,j), v(i,j), h(i-1,j), v(i,j-1),
    # d(i-1,j), d(i,j-1)) are (+, -, -, +, -, +)
    Bb = B[:, 2:]
    _, _, vt = np.linalg.svd(Bb)
    z = vt[-1]
    assert np.abs(Bb @ z).max() < 1e-12
    z = z / z[0]
    assert np.array_equal(np.sign(np.round(z, 12)), [1, -1, -1, 1, -1, 1])


def test_tiny_direct_solve():
    n = 4
    m, prm, A = build(n=n, lam=5.0, mu=1.0, tau=1.0, alpha=1.0, inv_M=0.1, k=0.5)
    b = m.pack(synthetic.rhs(n, 3))
    fi = m.free_idx
    Ad = A[fi][:, fi].toarray()
    x = np.linalg.solve(Ad, b[fi])
    assert np.linalg.norm(Ad @ x - b[fi]) < 1e-12 * np.linalg.norm(b)
    # the free-DoF count of the layout (header of the C ABI)
    N = n
    assert len(fi) == 2 * (N - 1) ** 2 + (3 * N * N - 2 * N) + (3 * N * N + 2 * N) + 2 * N * N


@pytest.mark.parametrize("prm", [dict(lam=1.0, mu=1.0, tau=1.0, alpha=1.0, inv_M=1.0),
                                 dict(lam=1e4, mu=0.7, tau=0.5, alpha=0.9, inv_M=1e-2),
                                 dict(lam=1e6, mu=1.3, tau=2.0, alpha=1.1, inv_M=0.0)])
def test_apply_rows_matches_assembled_operator(prm):
    """fem.apply_rows (the row-at-a-time product used for sampled checks at sizes too large
    to assemble) equals the assembled operator's product on every row of an 8-cell grid,
    with a lognormal per-triangle K and three parameter sets; constrained rows give 0 and
    constrained entries of x are ignored."""
    n = 8
    m = Mesh(n)
    p = fem.Params(**prm)
    KL, KU = synthetic.lognormal_k(n, 1.5, 7)
    kl, ku = fem.kinv_from_k(KL, KU)
    A = fem.assemble(m, p, kl, ku)
    x = m.pack(synthetic.uniform_field(n, 11))
    x_dirty = x + 3.0 * m.fixed                     # garbage in the constrained slots
    rows = np.arange(m.ndof)
    got = fem.apply_rows(m, p, kl, ku, x_dirty, rows)
    want = A @ x
    scale = np.max(np.abs(want))
    assert np.max(np.abs(got - want)) <= 1e-13 * scale
    assert np.all(got[m.fixed] == 0.0)


def test_exact_divdiv_element_dominates_reduced_quadrature():
    """The exactly integrated grad-div element matrix D = (div phi_a, div phi_b) (Sec. 2.1)
    and its reduced-quadrature form g g^T / |T| (Sec. 2.3): the divergence of P1 + bubble is
    linear on a triangle, so D has rank 3, D - g g^T / |T| is positive semidefinite (Cauchy-
    Schwarz), and the two agree on P1 fields (constant divergence)."""
    for tri in fem.reference_triangles(8).values():
        parts = fem.element_parts(tri)
        D, g, area = parts["Ddiv"], parts["g"], parts["area"]
        assert np.linalg.matrix_rank(D, tol=1e-12 * np.abs(D).max()) == 3
        ev = np.linalg.eigvalsh(D - np.outer(g, g) / area)
        assert ev.min() > -1e-12 * np.abs(D).max()
        P1 = np.zeros((9, 6))
        P1[:6, :6] = np.eye(6)
        diff = P1.T @ (D - np.outer(g, g) / area) @ P1
        assert np.abs(diff).max() <= 1e-12 * np.abs(D).max()
