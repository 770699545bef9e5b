"""Exact Braess-Sarazin relaxation on the GPU (smoother "bsr_exact": Sec. 3.2.2, Eq. bsr_p with
the fixed-stress S solved, not relaxed) against the oracle's exact BSR (sparse LU of S).

The GPU solves S dp = B z - r_p by preconditioned CG (a multigrid V-cycle on the coarser
levels' S, Jacobi on the last smoothing level) to a relative residual of 1e-11,
so dp carries a relative error up to kappa(S) 1e-11; the V-cycle tolerance is 1e-9 (the FP64
V-cycle parity bound) plus 10 kappa(S) 1e-11 with kappa(S) of the finest level computed here
from the oracle's S (coarser levels have smaller kappa).

* V-cycle parity, n = 16 and 32, constant and lognormal K, lambda = 1 and 1e4.
* FGMRES parity: the same 1e-8 true residual, counts within one, solutions within 1e-6.
* The CG count reported by the hierarchy is positive and below the number of P0 unknowns.
* A zero residual gives a zero correction (the CG stops before its first step).
* FP32 hierarchies with exact BSR are refused.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import synthetic
from oracle import fem, krylov, mg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bmg():
    import torch
    import paper_2107_04060_gb300 as m
    torch.cuda.set_device(0)
    return m


def dev(bmg, n, fields):
    import torch
    return torch.from_numpy(bmg.pack(n, fields)).cuda()


def to_oracle(bmg, mesh, t):
    return mesh.pack(bmg.unpack(mesh.n, t.double().cpu().numpy()))


def kappa_S(H, p):
    """2-norm condition number of the finest level's fixed-stress S (oracle matrices)."""
    L = H.levels[0]
    sm = L.smoother
    c_fs = p["inv_M"] + p["alpha"] ** 2 / (p["lam"] + p["mu"])
    S = (sp.diags(np.where(sm.mp_, c_fs * 0.5 * L.mesh.h ** 2, 0.0)) +
         sm.Bw @ sp.diags(sm.inv_tauDw) @ sm.Bw.T).tocsr()[sm.pidx][:, sm.pidx].toarray()
    ev = np.linalg.eigvalsh(S)
    return ev[-1] / ev[0]


def setup(bmg, n, p, kL, kU, omega=0.7):
    import torch
    Kf = None if kL is None else torch.from_numpy(bmg.pack_k(n, kL, kU)).cuda()
    s = bmg.assemble(n, p["lam"], p["mu"], Kf, 1.0, p["tau"], p["alpha"], p["inv_M"])
    h = bmg.setup_hierarchy(s, "bsr_exact", 1, 1, omega=omega, n_coarse=8)
    kinvL = np.ones((n, n)) if kL is None else 1 / kL
    kinvU = np.ones((n, n)) if kU is None else 1 / kU
    H = mg.Hierarchy(n, fem.Params(**p), kinvL, kinvU, smoother="bsr", omega=omega, n_coarse=8,
                     bsr_exact=True)
    return s, h, H


@pytest.mark.parametrize("n", [16, 32])
@pytest.mark.parametrize("lam", [1.0, 1e4])
@pytest.mark.parametrize("kind", ["const", "lognormal"])
def test_vcycle_parity(bmg, n, lam, kind):
    import torch
    p = dict(lam=lam, mu=1.0, tau=1.0, alpha=1.0, inv_M=1.0)
    kL, kU = (None, None) if kind == "const" else synthetic.lognormal_k(n, 1.0, 3)
    s, h, H = setup(bmg, n, p, kL, kU)
    f = synthetic.rhs(n, 5)
    r = dev(bmg, n, f)
    z = torch.empty_like(r)
    h.vcycle(r, z)
    zo = H.vcycle(H.levels[0].mesh.pack(f))
    zg = to_oracle(bmg, H.levels[0].mesh, z)
    tol = 1e-9 + 10 * kappa_S(H, p) * 1e-11
    assert np.abs(zg - zo).max() <= tol * np.abs(zo).max()
    it = h.schur_iters()
    assert 0 < it < 2 * n * n


def test_fgmres_parity(bmg):
    import torch
    n = 32
    p = dict(lam=1e4, mu=1.0, tau=1.0, alpha=1.0, inv_M=1.0)
    kL, kU = synthetic.lognormal_k(n, 1.0, 7)
    s, h, H = setup(bmg, n, p, kL, kU)
    f = synthetic.rhs(n, 0)
    b = dev(bmg, n, f)
    x = torch.zeros_like(b)
    info = h.fgmres_solve(b, x, rtol=1e-8, restart=50, maxit=300)
    A = H.levels[0].A
    bo = H.levels[0].mesh.pack(f)
    xo, oinfo = krylov.fgmres(A, bo, H.vcycle, rtol=1e-8, restart=50, maxit=300)
    assert info["status"] == "converged" and oinfo["converged"]
    assert abs(info["iters"] - oinfo["iters"]) <= 1, (info["iters"], oinfo["iters"])
    xg = to_oracle(bmg, H.levels[0].mesh, x)
    assert np.linalg.norm(bo - A @ xg) <= 1e-8 * np.linalg.norm(bo) * 1.0001
    assert np.linalg.norm(xg - xo) <= 1e-6 * np.linalg.norm(xo)


def test_zero_residual_gives_zero_correction(bmg):
    import torch
    n = 16
    p = dict(lam=10.0, mu=1.0, tau=1.0, alpha=1.0, inv_M=1.0)
    s, h, H = setup(bmg, n, p, None, None)
    r = torch.zeros(bmg.vector_len(n), dtype=torch.float64, device="cuda")
    z = torch.full_like(r, 7.0)
    h.vcycle(r, z)
    assert float(z.abs().max()) == 0.0


def test_fp32_exact_bsr_is_refused(bmg):
    s = bmg.assemble(16, 10.0, 1.0, None, 1.0, 1.0, 1.0, 1.0)
    with pytest.raises(bmg.BmgError):
        bmg.setup_hierarchy(s, "bsr_exact", 1, 1, omega=0.7, n_coarse=8, precision="fp32")
