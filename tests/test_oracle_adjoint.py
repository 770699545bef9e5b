"""Pins of the oracle's adjoint gradients (CPU): central finite differences of
J(theta, lambda, mu) = ||p - p_obs||^2 with direct solves, on seeded random directions.

The finite-difference step h = 1e-5 gives a truncation error O(h^2) ~ 1e-10 relative and a
rounding error ~ eps * |J| / h ~ 1e-11 relative to the directional derivative's scale; the
tolerance 1e-6 leaves room for the conditioning of the solves."""
import numpy as np
import pytest

import synthetic
from oracle import adjoint, fem
from oracle.mesh import Mesh


@pytest.fixture(scope="module")
def problem():
    n = 8
    prm = fem.Params(lam=10.0, mu=1.3, tau=1.0, alpha=1.0, inv_M=1.0)
    kL, kU = synthetic.lognormal_k(n, 1.0, 2)
    thL, thU = np.log(kL), np.log(kU)
    rL, rU = synthetic.lognormal_k(n, 1.0, 1)                  # reference log-K for p_obs
    b = Mesh(n).pack(synthetic.rhs(n, 0))
    m = Mesh(n)
    x_obs = adjoint.direct_solve(fem.assemble(m, prm, 1 / rL, 1 / rU), m, b)
    p_obs = adjoint.pressure(m, x_obs)
    return n, prm, thL, thU, b, p_obs


def test_theta_gradient_matches_central_differences(problem):
    n, prm, thL, thU, b, p_obs = problem
    J, dth, _, _, _, _ = adjoint.misfit_gradients(n, prm, thL, thU, b, p_obs)
    rng = np.random.default_rng(3)
    h = 1e-5
    for _ in range(8):
        d = rng.standard_normal((2, n, n))
        jp = adjoint.misfit(n, prm, thL + h * d[0], thU + h * d[1], b, p_obs)
        jm = adjoint.misfit(n, prm, thL - h * d[0], thU - h * d[1], b, p_obs)
        fd = (jp - jm) / (2 * h)
        an = float(np.sum(dth * d))
        assert an == pytest.approx(fd, rel=1e-6, abs=1e-9 * J)


@pytest.mark.parametrize("which", ["lam", "mu"])
def test_lame_gradients_match_central_differences(problem, which):
    n, prm, thL, thU, b, p_obs = problem
    _, _, dlam, dmu, _, _ = adjoint.misfit_gradients(n, prm, thL, thU, b, p_obs)
    base = getattr(prm, which)
    h = 1e-6 * base

    def J(v):
        q = fem.Params(lam=prm.lam, mu=prm.mu, tau=prm.tau, alpha=prm.alpha, inv_M=prm.inv_M)
        setattr(q, which, v)
        return adjoint.misfit(n, q, thL, thU, b, p_obs)
    fd = (J(base + h) - J(base - h)) / (2 * h)
    an = dlam if which == "lam" else dmu
    assert an == pytest.approx(fd, rel=1e-5)
