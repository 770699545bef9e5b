"""Pins of the oracle's multigrid and Krylov solver against the paper (CPU only).

* Table 2: measured two-grid factor of additive Vanka V(2,2), h = 1/64, Dirichlet
  displacement, E = 3e4, alpha = 1, mu_f = 1, M = 1e6, tau = 1, K = kI:
  nu = 0.499, k = 1, omega = 0.72 -> rho_N = 0.596;  nu = 0.4, k = 1, omega = 0.80 -> 0.403.
* Table 3: inexact Braess-Sarazin V(1,1): nu = 0.49, k = 1, omega_J = 1.21, omega = 0.69
  -> rho_N = 0.757.
* Sec. 4.3: with omega = 0.9 additive Vanka diverges for nu > 0.2 (negative control).
* Table 4: FGMRES with a four-level V-cycle on the steady manufactured problem (h = 1/64,
  coarsest h = 1/8, tolerance 1e-6): the Vanka counts at nu = 0, 0.4, 0.499 and k = 1 and
  the smallest k are the printed ones plus one constant offset (3 or 4).
* Sec. 5.1 / Fig. 5: |u - u_h|_H1 = O(h), ||p - p_h||_L2 = O(h^2), u-errors independent of nu.
* FGMRES (Sec. 5.1) reaches the direct solution on small grids.

The paper's stopping test (consecutive factors within 1e-3) is applied after a transient of
50 iterations (reading: the printed factors are asymptotic; from a random start the factor
rises slowly and the test can fire early).  The paper's measured factors differ from its LFA
predictions by up to 0.03 (e.g. 0.705 vs 0.722); the pins use a tolerance of 0.02.  The paper does not state nu1/nu2 for
Table 4; V(2,2) (the smoothing of Table 2, whose omega it reuses) is the reading tested.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import synthetic
from oracle import fem, krylov, manufactured, mg
from oracle.mesh import Mesh


def paper_params(nu):
    return fem.Params.from_paper(3e4, nu, tau=1.0, alpha=1.0, inv_M=1e-6)


def two_grid(nu, k, smoother, omega, omega_J=1.0, nu_s=2, n=64):
    prm = paper_params(nu)
    kinv = np.full((n, n), 1.0 / k)
    H = mg.Hierarchy(n, prm, kinv, kinv, smoother=smoother, omega=omega, omega_J=omega_J,
                     nu1=nu_s, nu2=nu_s, n_coarse=n // 2)
    m = H.levels[0].mesh
    x0 = m.pack(synthetic.uniform_field(n, 1)) * m.free
    rho, _ = mg.two_grid_rho(H, x0, max_it=100, min_it=50)
    return rho


@pytest.mark.slow
def test_table2_vanka_nu0499():
    assert two_grid(0.499, 1.0, "vanka", 0.72) == pytest.approx(0.596, abs=0.02)


@pytest.mark.slow
def test_table2_vanka_nu04():
    assert two_grid(0.4, 1.0, "vanka", 0.80) == pytest.approx(0.403, abs=0.02)


@pytest.mark.slow
def test_table3_bsr_nu049():
    assert two_grid(0.49, 1.0, "bsr", 0.69, omega_J=1.21, nu_s=1) == pytest.approx(0.757, abs=0.02)


def test_vanka_omega09_diverges_for_large_nu():
    assert two_grid(0.45, 1.0, "vanka", 0.9, n=32) > 1.0


@pytest.mark.slow
def test_table4_iterations_vanka():
    """Table 4 (Vanka rows, FGMRES to 1e-6 with a four-level V-cycle, h = 1/64): the oracle
    reproduces the printed pattern up to one constant offset.  With V(2,2) and Table 2's
    omega_opt for each (nu, k), the counts over nu in {0, 0.4, 0.499} and k = 1 and the
    smallest k exceed the paper's by 3 or 4 in every entry (printed 18, 10; 9, 10; 13, 14),
    so the drop at nu = 0 for k <= 1e-8 (18 -> 10) and the flat rows are reproduced; the
    offset itself comes from a stopping or scaling detail the paper does not print (a stop on
    the preconditioned residual or one decade less reduction does not give one constant)."""
    n = 64
    cases = [(0.0, 1.0, 0.92, 18), (0.0, 1e-8, 0.88, 10), (0.4, 1.0, 0.80, 9),
             (0.4, 1e-10, 0.76, 10), (0.499, 1.0, 0.72, 13), (0.499, 1e-10, 0.74, 14)]
    off = []
    for nu, k, om, paper in cases:
        prm = paper_params(nu)
        kinv = np.full((n, n), 1.0 / k)
        H = mg.Hierarchy(n, prm, kinv, kinv, smoother="vanka", omega=om, nu1=2, nu2=2, n_coarse=8)
        L = H.levels[0]
        b = manufactured.rhs(L.mesh, prm)
        _, info = krylov.fgmres(L.A, b, H.vcycle, rtol=1e-6, restart=50, maxit=100)
        off.append(info["iters"] - paper)
    assert min(off) >= 2 and max(off) <= 5, off
    assert max(off) - min(off) <= 1, off


def test_convergence_rates():
    eu, ep = {}, {}
    for nu in (0.4, 0.499):
        prm = paper_params(nu)
        for n in (8, 16, 32):
            m = Mesh(n)
            kinv = np.full((n, n), 1e6)                      # k = 1e-6 (Sec. 5.1)
            A = fem.assemble(m, prm, kinv, kinv)
            b = manufactured.rhs(m, prm)
            fi = m.free_idx
            x = np.zeros(m.ndof)
            x[fi] = spla.spsolve(A[fi][:, fi].tocsc(), b[fi])
            eu[nu, n], ep[nu, n] = manufactured.errors(m, x)
    for nu in (0.4, 0.499):
        for n in (8, 16):
            assert np.log2(eu[nu, n] / eu[nu, 2 * n]) == pytest.approx(1.0, abs=0.15)
            assert np.log2(ep[nu, n] / ep[nu, 2 * n]) > 1.85
    for n in (8, 16, 32):
        assert eu[0.4, n] == pytest.approx(eu[0.499, n], rel=0.02)
        assert ep[0.499, n] < ep[0.4, n]


@pytest.mark.parametrize("smoother,omega", [("vanka", 0.8), ("bsr", 0.7)])
def test_fgmres_reaches_direct_solution(smoother, omega):
    n = 16
    prm = fem.Params(lam=1.0, mu=1.0, tau=1.0, alpha=1.0, inv_M=1.0)
    kL, kU = synthetic.lognormal_k(n, 1.0, 5)
    H = mg.Hierarchy(n, prm, 1 / kL, 1 / kU, smoother=smoother, omega=omega, n_coarse=8)
    L = H.levels[0]
    b = L.mesh.pack(synthetic.rhs(n, 0))
    x, info = krylov.fgmres(L.A, b, H.vcycle, rtol=1e-11, restart=50, maxit=200)
    assert info["converged"]
    fi = L.mesh.free_idx
    xd = np.zeros_like(b)
    xd[fi] = spla.spsolve(L.A[fi][:, fi].tocsc(), b[fi])
    assert np.linalg.norm(x - xd) <= 1e-8 * np.linalg.norm(xd)


def test_fgmres_exact_preconditioner_one_iteration():
    n = 8
    m = Mesh(n)
    prm = fem.Params(lam=2.0, mu=1.0, tau=1.0, alpha=1.0, inv_M=1.0)
    one = np.ones((n, n))
    A = fem.assemble(m, prm, one, one)
    fi = m.free_idx
    lu = spla.splu(A[fi][:, fi].tocsc())

    def exact(v):
        z = np.zeros_like(v)
        z[fi] = lu.solve(v[fi])
        return z
    b = m.pack(synthetic.rhs(n, 2))
    _, info = krylov.fgmres(A, b, exact, rtol=1e-10)
    assert info["iters"] == 1


def test_galerkin_coarse_rt0_mass_matches_rediscretisation_for_constant_k():
    n = 16
    prm = fem.Params(lam=3.0, mu=1.0, tau=0.5, alpha=1.0, inv_M=1.0)
    kinv = np.full((n, n), 2.5)
    H = mg.Hierarchy(n, prm, kinv, kinv, smoother="vanka", omega=0.8, n_coarse=8)
    c = H.levels[1]
    direct = fem.assemble(c.mesh, prm, np.full((8, 8), 2.5), np.full((8, 8), 2.5))
    assert abs(c.A - direct).max() < 1e-12 * abs(direct).max()


def test_patch_shift_equals_compressibility():
    """Sec. 5.3 regularisation (1/M = 0): Vanka patch matrices of the system with 1/M = 0,
    shifted by p_shift = s, are exactly the patch matrices of the system with 1/M = s
    (reading: the shift is -s |T| on each P0 diagonal entry, the sign and scale of the
    -(1/M) M_p block).  Without the shift an interior patch is singular: constant pressure
    on the patch lies in the null space of its divergence rows."""
    from oracle.smoothers import Vanka
    n, s = 8, 1e-3
    m = Mesh(n)
    KL, KU = synthetic.lognormal_k(n, 1.0, 3)
    kl, ku = fem.kinv_from_k(KL, KU)
    base = dict(lam=1e4, mu=1.0, tau=1.0, alpha=1.0)
    A0 = fem.assemble(m, fem.Params(inv_M=0.0, **base), kl, ku)
    As = fem.assemble(m, fem.Params(inv_M=s, **base), kl, ku)
    v_shift = Vanka(A0, m, 1.0, p_shift=s)
    v_comp = Vanka(As, m, 1.0)
    assert len(v_shift.groups) == len(v_comp.groups)
    for (i1, inv1), (i2, inv2) in zip(v_shift.groups, v_comp.groups):
        assert np.array_equal(i1, i2)
        assert np.allclose(inv1, inv2, rtol=1e-12, atol=0.0)
    # unshifted interior patch at 1/M = 0: singular to working precision
    p = m.vertex_patch(4, 4)
    P = A0[p][:, p].toarray()
    assert np.linalg.cond(P) > 1e12
    assert np.linalg.cond(P - s * 0.5 * m.h ** 2 * np.diag(fem.type_mask(m, fem.P_TYPES)[p])) < 1e10


def test_w_cycle_restores_the_two_grid_factor_for_inexact_bsr():
    """The discussion of Table 4: multilevel inexact BSR struggles where the two-level method
    is robust, and W-cycles may be needed.  With the unit parameters (lambda = mu = K = tau =
    alpha = 1/M = 1) on a 32-cell grid, the stationary V(1,1) iteration with three levels
    diverges, while the W(1,1) iteration converges at the two-grid factor (within 0.03) and
    the LFA prediction for these parameters (0.687)."""
    n = 32
    prm = fem.Params(lam=1.0, mu=1.0, tau=1.0, alpha=1.0, inv_M=1.0)
    one = np.ones((n, n))

    def factor(nc, gamma):
        H = mg.Hierarchy(n, prm, one, one, smoother="bsr", omega=0.7, omega_J=1.0, n_coarse=nc,
                         gamma=gamma)
        L = H.levels[0]
        x = L.mesh.pack(synthetic.uniform_field(n, 1)) * L.mesh.free
        r0 = np.linalg.norm(L.A @ x)
        for _ in range(30):
            x = x + H.vcycle(-(L.A @ x))
            r1 = np.linalg.norm(L.A @ x)
            rho, r0 = r1 / r0, r1
        return rho

    tg = factor(16, 1)
    assert factor(8, 1) > 1.0
    w = factor(8, 2)
    assert abs(w - tg) < 0.03
    assert abs(w - 0.687) < 0.03


def test_exact_bsr_pressure_step_inverts_the_fixed_stress_schur_complement():
    """Sec. 3.2.2, Eq. bsr_p with S solved exactly: the exact-BSR correction d = (dy, dp) of a
    residual r satisfies the block system with the fixed-stress S built here from its
    definition, (1/M + alpha^2/(lambda + mu)) |T| on the P0 diagonal plus
    (tau B_w) (tau D_w)^{-1} (tau B_w)^T, with (tau B_w) and tau D_w read off the assembled
    operator:  F dy + B^T dp = r_y  and  S dp = B F^{-1} r_y - r_p.  F^{-1} is the smoother's
    displacement/flux solve, taken as a dense matrix from unit vectors.  Inexact BSR (one
    Jacobi sweep on S) fails the second identity."""
    n = 4
    prm = fem.Params(lam=50.0, mu=1.3, tau=0.5, alpha=0.9, inv_M=0.3)
    m = Mesh(n)
    kinv = np.linspace(0.5, 2.0, n * n).reshape(n, n)
    A = fem.assemble(m, prm, kinv, 1.0 / kinv[::-1]).tocsr()
    fr = np.nonzero(m.free)[0]
    pm = fem.type_mask(m, fem.P_TYPES)
    wm = fem.type_mask(m, fem.W_TYPES) & m.free
    yi = np.array([i for i in fr if not pm[i]])
    pi = np.nonzero(pm)[0]
    Ad = A.toarray()
    B = Ad[np.ix_(pi, yi)]
    Bw = Ad[np.ix_(pi, np.nonzero(wm)[0])]
    Dw = np.diag(Ad)[wm]
    area = 0.5 * m.h ** 2
    S = (prm.inv_M + prm.alpha ** 2 / (prm.lam + prm.mu)) * area * np.eye(len(pi)) + Bw @ np.diag(1 / Dw) @ Bw.T
    rng = np.random.default_rng(3)
    for exact in (True, False):
        sm = mg.BraessSarazin(A, m, prm, 0.7, 1.0, exact=exact)
        Finv = np.zeros((len(yi), len(yi)))
        for c, i in enumerate(yi):
            e = np.zeros(m.ndof)
            e[i] = 1.0
            Finv[:, c] = sm.F_inv(e)[yi]
        r = np.zeros(m.ndof)
        r[fr] = rng.standard_normal(len(fr))
        d = sm.correction(r)
        dy, dp = d[yi], d[pi]
        F = np.linalg.inv(Finv)
        assert np.abs(F @ dy + B.T @ dp - r[yi]).max() <= 1e-9 * np.abs(r).max()
        err = np.abs(S @ dp - (B @ Finv @ r[yi] - r[pi])).max() / np.abs(S @ dp).max()
        if exact:
            assert err <= 1e-10
        else:
            assert err > 1e-3
