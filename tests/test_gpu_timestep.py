"""Backward-Euler time stepping on the GPU (bmg_backward_euler_rhs + bmg_fgmres_solve, Sec.
2.1 Eqs. discrete1-3) against the oracle's time loop (oracle/timedep.py).

* The right-hand side of a step (loads plus the pressure-row history term) against the
  oracle's, element by element, for seeded vectors: 1e-13 relative (the same few FP64
  products per row on both sides).
* Six steps of the smooth manufactured problem (n = 16, tau = 1/64, lognormal-free K = 1e-2):
  the GPU's FGMRES (Vanka V(1,1), rtol 1e-11, warm-started from the previous step) against
  the oracle's direct solves, every step within 1e-7 relative, and the same final-time
  errors to 1e-6 relative.
"""
import numpy as np
import pytest

import synthetic
from oracle import fem, timedep
from oracle.mesh import Mesh

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bmg():
    import torch
    import paper_2107_04060_gb300 as m
    torch.cuda.set_device(0)
    return m


def dev(bmg, n, x_oracle, mesh):
    import torch
    return torch.from_numpy(bmg.pack(n, mesh.unpack(x_oracle))).cuda()


def to_oracle(bmg, mesh, t):
    return mesh.pack(bmg.unpack(mesh.n, t.double().cpu().numpy()))


@pytest.mark.parametrize("n", [5, 16])
def test_backward_euler_rhs_parity(bmg, n):
    import torch
    prm = fem.Params(lam=30.0, mu=1.3, tau=0.25, alpha=0.8, inv_M=0.5)
    kL, kU = synthetic.lognormal_k(n, 1.0, 3)
    K = torch.from_numpy(bmg.pack_k(n, kL, kU)).cuda()
    s = bmg.assemble(n, prm.lam, prm.mu, K, 0.0, prm.tau, prm.alpha, prm.inv_M)
    m = Mesh(n)
    A = fem.assemble(m, prm, 1 / kL, 1 / kU)
    xp = m.pack(synthetic.uniform_field(n, 5))
    ld = m.pack(synthetic.uniform_field(n, 6))
    b = torch.empty_like(dev(bmg, n, xp, m))
    s.backward_euler_rhs(dev(bmg, n, xp, m), dev(bmg, n, ld, m), b)
    want = ld * m.free + timedep.history(A, m, xp)
    got = to_oracle(bmg, m, b)
    assert np.abs(got - want).max() <= 1e-13 * np.abs(want).max()


def test_time_loop_matches_oracle(bmg):
    import torch
    n, steps = 16, 6
    K = 1e-2
    prm = fem.Params(lam=1e2, mu=1.0, tau=1.0 / 64, alpha=1.0, inv_M=1.0)
    mesh, A, xs = timedep.run(n, prm, K, steps)
    s = bmg.assemble(n, prm.lam, prm.mu, None, K, prm.tau, prm.alpha, prm.inv_M)
    h = bmg.setup_hierarchy(s, "vanka", 1, 1, omega=0.7, n_coarse=8)
    x = dev(bmg, n, xs[0], mesh)
    b = torch.empty_like(x)
    for mstep in range(1, steps + 1):
        ld = dev(bmg, n, timedep.loads(mesh, prm, K, mstep * prm.tau), mesh)
        s.backward_euler_rhs(x, ld, b)
        xn = x.clone()                                  # warm start from the previous step
        info = h.fgmres_solve(b, xn, rtol=1e-11, maxit=400, x0_is_zero=False)
        assert info["status"] == "converged"
        x = xn
        xo = xs[mstep]
        xg = to_oracle(bmg, mesh, x)
        assert np.linalg.norm(xg - xo) <= 1e-7 * np.linalg.norm(xo), mstep
    eg = timedep.errors(mesh, to_oracle(bmg, mesh, x), steps * prm.tau)
    eo = timedep.errors(mesh, xs[-1], steps * prm.tau)
    assert eg == pytest.approx(eo, rel=1e-6)
