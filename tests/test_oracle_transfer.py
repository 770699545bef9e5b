"""Pins of the oracle's grid transfers (CPU only).

* App. B restriction-symbol coefficients, read as couplings of P (reading: the bubble block
  printed in App. B is P-oriented, rows = fine types): 1/4, sqrt2/8, 5 sqrt2/8, -1 between
  bubbles; 3 sqrt2/16 and 3/8 from P1 to bubbles; sqrt2/2, 1 from bubbles to P1; the 7-point
  P1 weights 1 and 1/2; the RT0 weights of R_w (2 c3 + c4, sqrt2 c2, sqrt2/2 c3, ...);
* the defining property of P_u (Sec. 3.1, Eq. divfreefine): every column has zero net flux
  through every corner child, so B_u,h P_u = Q B_u,H (Q: injection into the interior
  child), hence P_p^T B_u,h P_u = B_u,H and P_u^T (B^T M^{-1} B)_h P_u = 4 (B^T M^{-1} B)_H;
* nested-space Galerkin identities for the canonical RT0 / P0 interpolation:
  P_w^T M_w,h P_w = M_w,H,  P_p^T B_w,h P_w = B_w,H,  P_p^T M_p,h P_p = M_p,H.
"""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import fem, transfer
from oracle.mesh import Mesh

S2 = np.sqrt(2.0)


@pytest.fixture(scope="module")
def P48():
    c, f = Mesh(4), Mesh(8)
    return c, f, transfer.prolongation(f, c).tocsc()


def column(P, f, c, t, I, J):
    col = P[:, c.idx(t, I, J)]
    out = {}
    for k, v in zip(col.indices, col.data):
        for tt in f.offsets:
            o = f.offsets[tt]
            r, cc = f.shapes[tt]
            if o <= k < o + r * cc:
                jj, ii = divmod(k - o, cc)
                out[(tt, ii, jj)] = v
    return out


def test_appendix_b_bubble_couplings(P48):
    c, f, P = P48
    d = column(P, f, c, "bd", 1, 1)
    assert d[("bd", 3, 2)] == pytest.approx(0.25) and d[("bd", 2, 3)] == pytest.approx(0.25)
    for key in [("bh", 2, 3), ("bh", 3, 3), ("bv", 3, 2), ("bv", 3, 3)]:
        assert d[key] == pytest.approx(5 * S2 / 8, rel=1e-13)
    assert d[("ux", 3, 3)] == pytest.approx(S2 / 2) and d[("uy", 3, 3)] == pytest.approx(S2 / 2)
    hcol = column(P, f, c, "bh", 1, 2)
    assert hcol[("bh", 2, 4)] == pytest.approx(0.25) and hcol[("bh", 3, 4)] == pytest.approx(0.25)
    assert hcol[("bv", 3, 3)] == pytest.approx(-1.0) and hcol[("bv", 3, 4)] == pytest.approx(-1.0)
    assert hcol[("bd", 3, 3)] == pytest.approx(S2 / 8) and hcol[("bd", 2, 4)] == pytest.approx(S2 / 8)
    assert hcol[("uy", 3, 4)] == pytest.approx(1.0) and ("ux", 3, 4) not in hcol


def test_appendix_b_p1_couplings(P48):
    c, f, P = P48
    u = column(P, f, c, "ux", 2, 2)
    p1 = {k: v for k, v in u.items() if k[0] == "ux"}
    assert p1[("ux", 4, 4)] == pytest.approx(1.0)
    half = [(5, 4), (3, 4), (4, 5), (4, 3), (5, 3), (3, 5)]        # 7-point, anti-diagonal
    for (ii, jj) in half:
        assert p1[("ux", ii, jj)] == pytest.approx(0.5)
    assert len(p1) == 7
    bub = sorted(round(v, 12) for k, v in u.items() if k[0].startswith("b"))
    assert bub == sorted([round(x, 12) for x in [-3 * S2 / 16, -3 * S2 / 16, 3 * S2 / 16, 3 * S2 / 16]
                          + [-3 / 8] * 4 + [3 / 8] * 4])


def test_appendix_b_rt0_couplings(P48):
    c, f, P = P48
    w = column(P, f, c, "wd", 1, 1)
    assert w[("wd", 3, 2)] == pytest.approx(1.0) and w[("wd", 2, 3)] == pytest.approx(1.0)
    assert w[("wd", 2, 2)] == pytest.approx(0.5) and w[("wd", 3, 3)] == pytest.approx(0.5)
    for key in [("wh", 2, 3), ("wh", 3, 3), ("wv", 3, 2), ("wv", 3, 3)]:
        assert w[key] == pytest.approx(S2 / 2)
    wh = column(P, f, c, "wh", 1, 2)
    assert wh[("wh", 2, 4)] == pytest.approx(1.0) and wh[("wh", 3, 4)] == pytest.approx(1.0)
    assert wh[("wh", 3, 3)] == pytest.approx(0.5) and wh[("wh", 2, 5)] == pytest.approx(0.5)
    assert wh[("wd", 3, 3)] == pytest.approx(S2 / 4) and wh[("wd", 2, 4)] == pytest.approx(S2 / 4)


def _blocks(n):
    m = Mesh(n)
    prm = fem.Params(lam=1.0, mu=1.0, tau=1.0, alpha=1.0, inv_M=1.0)
    one = np.ones((n, n))
    A = fem.assemble(m, prm, one, one)
    u = fem.type_mask(m, fem.U_TYPES)
    w = fem.type_mask(m, fem.W_TYPES)
    p = fem.type_mask(m, fem.P_TYPES)
    return m, A, u, w, p


def test_divergence_preserving_identities():
    f, Af, uf, wf, pf = _blocks(8)
    c, Ac, uc, wc, pc = _blocks(4)
    P = transfer.prolongation(f, c).tocsr()
    Pu = P[uf][:, uc]
    Pp = P[pf][:, pc]
    Buf = Af[pf][:, uf]                                   # alpha B_u, alpha = 1
    Buc = Ac[pc][:, uc]
    # zero flux through every corner child: B_h P_u has nonzeros only on interior children
    BP = (Buf @ Pu).toarray()
    Q = np.zeros((BP.shape[0], Buc.shape[0]))
    for o, I, J in c.triangles():
        kids = transfer.fine_triangle([(2 * I + 1, 2 * J + 1), (2 * I, 2 * J + 1), (2 * I + 1, 2 * J)]) \
            if o == "L" else transfer.fine_triangle([(2 * I + 1, 2 * J + 1), (2 * I + 2, 2 * J + 1), (2 * I + 1, 2 * J + 2)])
        fo, fi, fj = kids
        rf = f.idx("pL" if fo == "L" else "pU", fi, fj) - f.offsets["pL"]
        rc = c.idx("pL" if o == "L" else "pU", I, J) - c.offsets["pL"]
        Q[rf, rc] = 1.0
    assert np.allclose(BP, Q @ Buc.toarray(), atol=1e-13)
    assert np.allclose((Pp.T @ Buf @ Pu).toarray(), Buc.toarray(), atol=1e-13)
    hf = 1.0 / 8
    hc = 1.0 / 4
    Gf = Buf.T @ sp.diags(np.full(Buf.shape[0], 2.0 / hf ** 2)) @ Buf
    Gc = Buc.T @ sp.diags(np.full(Buc.shape[0], 2.0 / hc ** 2)) @ Buc
    assert np.allclose((Pu.T @ Gf @ Pu).toarray(), 4.0 * Gc.toarray(), atol=1e-11)


def test_nested_galerkin_identities():
    f, Af, uf, wf, pf = _blocks(8)
    c, Ac, uc, wc, pc = _blocks(4)
    P = transfer.prolongation(f, c).tocsr()
    Pw = P[wf][:, wc]
    Pp = P[pf][:, pc]
    assert np.allclose((Pw.T @ Af[wf][:, wf] @ Pw).toarray(), Ac[wc][:, wc].toarray(), atol=1e-13)
    assert np.allclose((Pp.T @ Af[pf][:, wf] @ Pw).toarray(), Ac[pc][:, wc].toarray(), atol=1e-13)
    assert np.allclose((Pp.T @ Af[pf][:, pf] @ Pp).toarray(), Ac[pc][:, pc].toarray(), atol=1e-13)


def test_divergence_free_maps_to_divergence_free():
    f, Af, uf, wf, pf = _blocks(8)
    c, Ac, uc, wc, pc = _blocks(4)
    P = transfer.prolongation(f, c).tocsr()
    Buc = Ac[pc][:, uc].toarray()
    _, s, vt = np.linalg.svd(Buc)
    null = vt[np.sum(s > 1e-12 * s[0]):]                 # coarse div-free displacements
    assert null.shape[0] > 0
    fine = P[uf][:, uc] @ null.T
    assert np.abs(Af[pf][:, uf] @ fine).max() < 1e-12


def test_restriction_is_transpose(P48):
    c, f, P = P48
    R = transfer.restriction(P.tocsr())
    assert abs(R - P.T).max() == 0.0
