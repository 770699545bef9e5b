"""Adjoint gradients on the GPU (bmg_adjoint_gradient through the differentiable solve):
against the CPU oracle's adjoint (direct solves) and against central finite differences of
J = ||p - p_obs||^2 on 32 seeded random directions of theta (the configuration's check), at
solver tolerance 1e-12.  The tolerances follow from that solver tolerance: gradients
agree with the oracle to ~1e-9 relative; finite differences with step 1e-4 carry an
O(h^2) truncation error ~1e-8 relative plus a solve error ~1e-12 |J| / h."""
import numpy as np
import pytest

import synthetic
from oracle import adjoint, fem
from oracle.mesh import Mesh

pytestmark = pytest.mark.gpu


def setup(n=16, lam=10.0, mu=1.3):
    import torch
    import paper_2107_04060_gb300 as bmg
    torch.cuda.set_device(0)
    kL, kU = synthetic.lognormal_k(n, 1.0, 2)
    rL, rU = synthetic.lognormal_k(n, 1.0, 1)
    prm = fem.Params(lam=lam, mu=mu, tau=1.0, alpha=1.0, inv_M=1.0)
    m = Mesh(n)
    bo = m.pack(synthetic.rhs(n, 0))
    p_obs = adjoint.pressure(m, adjoint.direct_solve(fem.assemble(m, prm, 1 / rL, 1 / rU), m, bo))
    theta = torch.from_numpy(np.stack([np.log(kL), np.log(kU)]).astype(np.float32)).cuda()
    b = torch.from_numpy(bmg.pack(n, synthetic.rhs(n, 0))).cuda()
    return bmg, prm, m, bo, theta, b, torch.from_numpy(p_obs).cuda()


def loss(theta, lam, mu, b, p_obs, **cfg):
    from paper_2107_04060_gb300.differentiable import pressure_solve
    p = pressure_solve(theta, lam, mu, b, rtol=1e-12, maxit=4000, **cfg)
    return ((p - p_obs) ** 2).sum()


def test_adjoint_matches_oracle():
    import torch
    bmg, prm, m, bo, theta, b, p_obs = setup()
    th = theta.clone().requires_grad_(True)
    lam = torch.tensor(prm.lam, dtype=torch.float64, requires_grad=True)
    mu = torch.tensor(prm.mu, dtype=torch.float64, requires_grad=True)
    J = loss(th, lam, mu, b, p_obs)
    J.backward()
    thn = theta.double().cpu().numpy()
    Jo, dth, dlam, dmu, _, _ = adjoint.misfit_gradients(m.n, prm, thn[0], thn[1], bo, p_obs.cpu().numpy())
    assert J.item() == pytest.approx(Jo, rel=1e-9)
    g = th.grad.double().cpu().numpy()
    assert np.abs(g - dth).max() <= 1e-6 * np.abs(dth).max()
    assert lam.grad.item() == pytest.approx(dlam, rel=1e-6)
    assert mu.grad.item() == pytest.approx(dmu, rel=1e-6)


def test_adjoint_matches_central_differences_32_directions():
    import torch
    bmg, prm, m, bo, theta, b, p_obs = setup()
    lam = torch.tensor(prm.lam, dtype=torch.float64)
    mu = torch.tensor(prm.mu, dtype=torch.float64)
    th64 = theta.double()
    th = th64.float().clone().requires_grad_(True)
    J = loss(th, lam, mu, b, p_obs)
    J.backward()
    g = th.grad.double()
    rng = np.random.default_rng(3)
    h = 1e-4
    worst = 0.0
    for _ in range(32):
        d = torch.from_numpy(rng.standard_normal((2, m.n, m.n))).cuda()
        # theta is float32: perturb in float64 and round, then use the realised step
        tp = (th64 + h * d).float()
        tm = (th64 - h * d).float()
        jp = loss(tp, lam, mu, b, p_obs).item()
        jm = loss(tm, lam, mu, b, p_obs).item()
        dd = (tp.double() - tm.double()) / 2.0
        fd = (jp - jm) / 2.0
        an = float((g * dd).sum())
        worst = max(worst, abs(an - fd) / max(abs(fd), 1e-12 * J.item()))
    assert worst < 1e-4, worst


def test_gradient_kernel_full_size_matches_oracle():
    """The adjoint workload's size (1024 x 1024): given the GPU's forward and adjoint
    solutions, the gradient kernel agrees with the oracle's element-wise gradient formulas
    evaluated on the same x and xi: dL/dtheta per triangle to 1e-12 of its maximum;
    dL/dlambda and dL/dmu are sums of 2M terms of both signs, reduced in a fixed tree of CTA
    partials on one side and by numpy's pairwise summation on the other, so their difference
    is bounded by about N eps sum|t_T| (N = 2M, eps = 1.1e-16): 1e-8 relative covers a sum of
    magnitudes up to 40x the result."""
    import torch
    import paper_2107_04060_gb300 as bmg
    torch.cuda.set_device(0)
    n = 1024
    prm = fem.Params(lam=10.0, mu=1.3, tau=1.0, alpha=1.0, inv_M=1.0)
    kL, kU = synthetic.lognormal_k(n, 1.0, 2)
    theta = np.stack([np.log(kL), np.log(kU)]).astype(np.float32)
    P = bmg.pitch(n)
    th = torch.zeros(2, n + 1, P, dtype=torch.float32, device="cuda")
    th[:, :n, :n] = torch.from_numpy(theta).cuda()
    s = bmg.assemble_logk(n, prm.lam, prm.mu, th.reshape(-1), 1.0, 1.0, 1.0)
    h = bmg.setup_hierarchy(s, "vanka", 1, 1, omega=0.8)
    b = torch.from_numpy(bmg.pack(n, synthetic.rhs(n, 0))).cuda()
    x = torch.zeros_like(b)
    assert h.fgmres_solve(b, x, rtol=1e-8, maxit=1000)["status"] == "converged"
    gx = torch.zeros(10, n + 1, P, dtype=torch.float64, device="cuda")
    gx[8:10, :n, :n] = x.view(10, n + 1, P)[8:10, :n, :n]          # dL/dx for L = ||p||^2 / 2
    xi = torch.zeros_like(b)
    assert h.fgmres_solve(gx.reshape(-1), xi, rtol=1e-8, maxit=1000)["status"] == "converged"
    dth = torch.empty(2 * (n + 1) * P, dtype=torch.float64, device="cuda")
    dl = torch.empty(2, dtype=torch.float64, device="cuda")
    s.adjoint_gradient(x, xi, dth, dl)
    m = Mesh(n)
    xo = m.pack(bmg.unpack(n, x.cpu().numpy()))
    xio = m.pack(bmg.unpack(n, xi.cpu().numpy()))
    th64 = theta.astype(np.float64)
    do, dlo, dmo = adjoint.gradients(m, prm, th64[0], th64[1], xo, xio)
    dg = dth.view(2, n + 1, P)[:, :n, :n].cpu().numpy()
    assert np.abs(dg - do).max() <= 1e-12 * np.abs(do).max()
    assert dl[0].item() == pytest.approx(dlo, rel=1e-8)
    assert dl[1].item() == pytest.approx(dmo, rel=1e-8)
