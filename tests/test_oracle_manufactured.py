"""Pins of the steady manufactured problem of Sec. 5.1 (oracle/manufactured.py), each
against something other than the module itself:

* the exact displacement is the curl of phi = [x y (1-x)(1-y)]^2 and its gradient and
  -mu Laplace(u) are that field's derivatives: compared with sympy's differentiation of
  phi at seeded points (the module codes the derivatives by hand through F, F', F'', F''');
* the exact displacement is divergence-free and vanishes on the boundary of the square;
* Radon's 7-point rule integrates every monomial x^a y^b with a + b <= 5 exactly over a
  triangle (closed form a! b! / (a + b + 2)! on the reference triangle, and affine images)
  and is not exact at degree 6;
* the load vector's P0 rows are -(1/M)|T|, and the natural boundary condition p = 1 loads
  only RT0 DoFs on the boundary, with opposite signs on opposite sides."""
import math

import numpy as np
import pytest

from oracle import fem, manufactured
from oracle.mesh import Mesh


def test_exact_field_matches_symbolic_derivatives():
    sp = pytest.importorskip("sympy")
    x, y = sp.symbols("x y")
    phi = (x * y * (1 - x) * (1 - y)) ** 2
    u = sp.Matrix([sp.diff(phi, y), -sp.diff(phi, x)])
    grad = u.jacobian([x, y])
    lap = sp.Matrix([sp.diff(u[k], x, 2) + sp.diff(u[k], y, 2) for k in range(2)])
    fu, fg, fl = (sp.lambdify((x, y), e, "numpy") for e in (u, grad, lap))
    mu = 1.7
    rng = np.random.default_rng(3)
    for px, py in rng.uniform(0, 1, (25, 2)):
        assert np.allclose(manufactured.exact_u(px, py), np.array(fu(px, py), float).ravel(),
                           rtol=1e-12, atol=1e-15)
        assert np.allclose(manufactured.exact_grad_u(px, py), np.array(fg(px, py), float),
                           rtol=1e-12, atol=1e-15)
        assert np.allclose(manufactured.body_force(px, py, mu), -mu * np.array(fl(px, py), float).ravel(),
                           rtol=1e-12, atol=1e-13)


def test_exact_field_is_divergence_free_and_zero_on_the_boundary():
    rng = np.random.default_rng(4)
    for px, py in rng.uniform(0, 1, (25, 2)):
        g = manufactured.exact_grad_u(px, py)
        assert abs(g[0, 0] + g[1, 1]) <= 1e-15
    for t in np.linspace(0, 1, 11):
        for px, py in ((t, 0.0), (t, 1.0), (0.0, t), (1.0, t)):
            assert np.all(manufactured.exact_u(px, py) == 0.0)


def _rule(X):
    """Radon's points and weights mapped to the triangle with vertices X (3 x 2)."""
    area = 0.5 * abs((X[1, 0] - X[0, 0]) * (X[2, 1] - X[0, 1]) - (X[2, 0] - X[0, 0]) * (X[1, 1] - X[0, 1]))
    pts = manufactured.RADON_BARY @ X
    return pts, manufactured.RADON_W * area


def test_radon_rule_is_exact_to_degree_five():
    assert math.isclose(manufactured.RADON_W.sum(), 1.0, rel_tol=1e-15)
    assert np.allclose(manufactured.RADON_BARY.sum(axis=1), 1.0)
    ref = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0]])
    pts, w = _rule(ref)
    for a in range(6):
        for b in range(6 - a):
            exact = math.factorial(a) * math.factorial(b) / math.factorial(a + b + 2)
            got = float(np.sum(w * pts[:, 0] ** a * pts[:, 1] ** b))
            assert math.isclose(got, exact, rel_tol=1e-13), (a, b, got, exact)
    # degree 6: x^6 over the reference triangle is 6!/8! = 1/56; the rule misses it
    got6 = float(np.sum(w * pts[:, 0] ** 6))
    assert abs(got6 - 1.0 / 56.0) > 1e-6
    # an affine image: integral of x^2 y over the triangle (0.2,0.1),(0.9,0.3),(0.4,0.8)
    sp = pytest.importorskip("sympy")
    X = np.array([[0.2, 0.1], [0.9, 0.3], [0.4, 0.8]])
    s, t = sp.symbols("s t")
    xs = X[0, 0] + (X[1, 0] - X[0, 0]) * s + (X[2, 0] - X[0, 0]) * t
    ys = X[0, 1] + (X[1, 1] - X[0, 1]) * s + (X[2, 1] - X[0, 1]) * t
    jac = abs((X[1, 0] - X[0, 0]) * (X[2, 1] - X[0, 1]) - (X[2, 0] - X[0, 0]) * (X[1, 1] - X[0, 1]))
    exact = float(sp.integrate(sp.integrate(xs ** 2 * ys * jac, (t, 0, 1 - s)), (s, 0, 1)))
    pts, w = _rule(X)
    assert math.isclose(float(np.sum(w * pts[:, 0] ** 2 * pts[:, 1])), exact, rel_tol=1e-13)


def test_load_vector_pressure_rows_and_boundary_flux_terms():
    n = 4
    m = Mesh(n)
    prm = fem.Params(lam=10.0, mu=1.0, tau=0.7, alpha=1.0, inv_M=2.5)
    b = manufactured.rhs(m, prm)
    area = 0.5 / n ** 2
    for o, i, j in m.triangles():
        assert math.isclose(b[m.tri_dofs(o, i, j)[12]], -prm.inv_M * area, rel_tol=1e-14)
    h = 1.0 / n
    for i in range(n):
        assert math.isclose(b[m.idx("wh", i, 0)], prm.tau * h, rel_tol=1e-14)
        assert math.isclose(b[m.idx("wh", i, n)], -prm.tau * h, rel_tol=1e-14)
        for j in range(1, n):
            assert b[m.idx("wh", i, j)] == 0.0          # interior edges carry no boundary load
    for j in range(n):
        assert math.isclose(b[m.idx("wv", 0, j)], prm.tau * h, rel_tol=1e-14)
        assert math.isclose(b[m.idx("wv", n, j)], -prm.tau * h, rel_tol=1e-14)
    # the boundary loads of p = 1 cancel: the outward flux of a constant pressure balances
    wsum = sum(b[m.idx("wh", i, jj)] for i in range(n) for jj in (0, n)) + \
        sum(b[m.idx("wv", ii, j)] for j in range(n) for ii in (0, n))
    assert abs(wsum) <= 1e-14
