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
