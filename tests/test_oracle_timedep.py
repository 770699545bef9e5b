"""Pins of the oracle's backward-Euler time stepping (oracle/timedep.py; Sec. 2.1 Eqs.
discrete1-3) on CPU.

* The loads against symbolic derivatives (sympy) of the exact fields: rho g = -div sigma(u)
  + alpha grad p, f = d/dt((1/M) p + alpha div u) + div w with w = -K grad p.
* Convergence of the final-time errors with tau = h^2: |u - u_h|_H1 first order and the
  pressure against its cell averages second order (the rates Sec. 5.1 states for the steady
  problem; backward Euler adds O(tau) = O(h^2)).
* A planted mistake: the history term with the wrong sign stops the pressure from
  converging.
"""
import numpy as np
import pytest

from oracle import fem, timedep

PRM = dict(lam=1e2, mu=1.0, alpha=1.0, inv_M=1.0)
K = 1e-2
T = 1.0 / 32


def test_loads_match_symbolic_derivatives():
    sympy = pytest.importorskip("sympy")
    x, y, t = sympy.symbols("x y t")
    mu, lam, al, invM, k = 1.3, 7.0, 0.9, 0.4, 0.05
    phi = (x * y * (1 - x) * (1 - y)) ** 2
    u = sympy.exp(-t) * sympy.Matrix([sympy.diff(phi, y), -sympy.diff(phi, x)])
    p = sympy.exp(-t) * sympy.sin(sympy.pi * x) * sympy.sin(sympy.pi * y)
    gu = u.jacobian([x, y])
    eps = (gu + gu.T) / 2
    divu = sympy.simplify(gu[0, 0] + gu[1, 1])
    sigma = 2 * mu * eps + lam * divu * sympy.eye(2)
    rhog = -sympy.Matrix([sympy.diff(sigma[0, 0], x) + sympy.diff(sigma[0, 1], y),
                          sympy.diff(sigma[1, 0], x) + sympy.diff(sigma[1, 1], y)]) \
        + al * sympy.Matrix([sympy.diff(p, x), sympy.diff(p, y)])
    w = -k * sympy.Matrix([sympy.diff(p, x), sympy.diff(p, y)])
    f = sympy.diff(invM * p + al * divu, t) + sympy.diff(w[0], x) + sympy.diff(w[1], y)
    prm = fem.Params(lam=lam, mu=mu, alpha=al, inv_M=invM)
    rng = np.random.default_rng(0)
    for xv, yv, tv in rng.uniform(0, 1, size=(5, 3)):
        sub = {x: xv, y: yv, t: tv}
        assert divu.subs(sub) == pytest.approx(0.0, abs=1e-12)
        got = timedep.u_force(xv, yv, tv, prm)
        want = np.array([float(rhog[0].subs(sub)), float(rhog[1].subs(sub))])
        assert np.allclose(got, want, rtol=1e-10, atol=1e-12)
        assert timedep.source_f(xv, yv, tv, prm, k) == pytest.approx(float(f.subs(sub)), rel=1e-10)
        assert timedep.exact_p(xv, yv, tv) == pytest.approx(float(p.subs(sub)), rel=1e-12)


def final_errors(n, history=None):
    tau = 1.0 / n ** 2
    steps = round(T / tau)
    prm = fem.Params(tau=tau, **PRM)
    mesh, A, xs = timedep.run(n, prm, K, steps)
    return timedep.errors(mesh, xs[-1], steps * tau)


def test_backward_euler_converges_at_the_stated_rates():
    (u8, p8), (u16, p16) = final_errors(8), final_errors(16)
    assert np.log2(u8 / u16) == pytest.approx(1.0, abs=0.2)
    assert np.log2(p8 / p16) == pytest.approx(2.0, abs=0.25)


def test_wrong_history_sign_is_caught(monkeypatch):
    good = timedep.history
    monkeypatch.setattr(timedep, "history", lambda A, mesh, x: -good(A, mesh, x))
    (u8, p8), (u16, p16) = final_errors(8), final_errors(16)
    assert np.log2(p8 / p16) < 1.0 or p16 > 1e-2
