"""Parity of the CUDA V-cycle and solver with the oracle on the kernel paths the bench runs.

The tile of every operator and smoother launch is chosen at setup by timing; grids of 128
and more cells per side get the large tiles (and, with uniform coefficients, the
symmetry-adapted interior patch solve) that the small-grid parity tests never reach.  Here
every candidate tile is forced in turn (BMG_FORCE_APPLY_TILE, BMG_FORCE_SMOOTHER_TILE) and
each V-cycle is compared with the oracle's, element by element.

Tolerances as in test_gpu_parity.py: 1e-9 relative (max-norm) for an FP64 V-cycle, whose
exactly inverted patch matrices amplify FP64 rounding differences of the two summation
orders; FP32-MG solutions within 1e-6 (2-norm) of the oracle's direct solution (both solve
to a 1e-8 true relative residual in FP64).
"""
import os

import numpy as np
import pytest

import synthetic
from oracle import fem, krylov, mg
from oracle.mesh import Mesh

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


def kfield(bmg, n, kL, kU):
    import torch
    return torch.from_numpy(bmg.pack_k(n, kL, kU)).cuda()


def relmax(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def setup_forced(bmg, s, smoother, omega, tile, apply_tile=None, **kw):
    """GPU hierarchy with the smoother tile forced to ``tile`` and the operator tile to
    ``apply_tile`` (default: ``tile``) on every level."""
    old = {k: os.environ.get(k) for k in ("BMG_FORCE_APPLY_TILE", "BMG_FORCE_SMOOTHER_TILE")}
    try:
        os.environ["BMG_FORCE_APPLY_TILE"] = str(tile if apply_tile is None else apply_tile)
        os.environ["BMG_FORCE_SMOOTHER_TILE"] = str(tile)
        return bmg.setup_hierarchy(s, smoother, 1, 1, omega=omega, omega_J=1.0, n_coarse=8, **kw)
    finally:
        for k, v in old.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


CASES = [("vanka", 0.8, "const"), ("vanka", 0.7, "lognormal"), ("bsr", 0.7, "const"),
         ("bsr", 0.7, "lognormal")]


@pytest.mark.parametrize("smoother,omega,kind", CASES)
def test_vcycle_parity_every_tile_n128(bmg, smoother, omega, kind):
    """n = 128 (five levels down to 8): every tile candidate of the operator and of the
    smoother, constant coefficients (symmetry-adapted interior Vanka solve) and lognormal K
    (per-patch inverses); the register-capped operator tiles 6 and 7, the operator tiles 8
    and 9 that load b first, and the smoothers' one-thread-per-patch candidates 5-7 with the
    32 x 8 operator tile."""
    import torch
    n = 128
    p = dict(lam=1.0, mu=1.0, tau=1.0, alpha=1.0, inv_M=1.0) if kind == "const" else \
        dict(lam=1e4, mu=1.0, tau=1.0, alpha=1.0, inv_M=1.0)
    if kind == "const":
        kL = kU = None
        kinvL = kinvU = np.ones((n, n))
    else:
        kL, kU = synthetic.lognormal_k(n, 1.0, 3)
        kinvL, kinvU = 1 / kL, 1 / kU
    Kf = None if kL is None else kfield(bmg, n, kL, kU)
    s = bmg.assemble(n, p["lam"], p["mu"], Kf, 1.0, p["tau"], p["alpha"], p["inv_M"])
    H = mg.Hierarchy(n, fem.Params(**p), kinvL, kinvU, smoother=smoother, omega=omega,
                     omega_J=1.0, nu1=1, nu2=1, n_coarse=8)
    f = synthetic.rhs(n, 5)
    zo = H.vcycle(H.levels[0].mesh.pack(f))
    r = dev(bmg, n, f)
    combos = [(t, t) for t in range(5)] + [(0, 6), (1, 7), (0, 8), (1, 9)]   # (smoother, operator)
    combos += [(5, 0), (6, 0), (7, 0)]                             # one thread per patch solve
    for tile, at in combos:
        h = setup_forced(bmg, s, smoother, omega, tile, apply_tile=at)
        key = "vanka" if smoother == "vanka" else "vanka_u"
        assert all(h.tile(l, key) == tile and h.tile(l, "apply") == at for l in range(h.levels - 1))
        z = torch.empty_like(r)
        h.vcycle(r, z)
        err = relmax(to_oracle(bmg, H.levels[0].mesh, z), zo)
        assert err < 1e-9, (tile, at, err)
        h.close()


@pytest.mark.parametrize("smoother,omega", [("vanka", 0.7), ("bsr", 0.7)])
def test_vcycle_parity_tuned_n256(bmg, smoother, omega):
    """n = 256 with the tiles the setup-time tuner picks (the bench's launch configuration on
    the second level of a 512 grid), lognormal K."""
    import torch
    n = 256
    p = dict(lam=1e4, mu=1.0, tau=1.0, alpha=1.0, inv_M=1.0)
    kL, kU = synthetic.lognormal_k(n, 1.0, 9)
    s = bmg.assemble(n, p["lam"], p["mu"], kfield(bmg, n, kL, kU), 1.0, p["tau"], p["alpha"], p["inv_M"])
    h = bmg.setup_hierarchy(s, smoother, 1, 1, omega=omega, omega_J=1.0, n_coarse=8)
    H = mg.Hierarchy(n, fem.Params(**p), 1 / kL, 1 / kU, smoother=smoother, omega=omega,
                     omega_J=1.0, nu1=1, nu2=1, n_coarse=8)
    f = synthetic.rhs(n, 6)
    r = dev(bmg, n, f)
    z = torch.empty_like(r)
    h.vcycle(r, z)
    zo = H.vcycle(H.levels[0].mesh.pack(f))
    assert relmax(to_oracle(bmg, H.levels[0].mesh, z), zo) < 1e-9


@pytest.mark.parametrize("n", [32, 128])
def test_vcycle_parity_incompressible_with_patch_shift(bmg, n):
    """1/M = 0 (the Sec. 5.3 setting) with the patch regularisation p_shift = s: the GPU
    V-cycle (which adds -s |T| to the P0 diagonal of every patch) against the oracle's with
    the same reading, lognormal K."""
    import torch
    p = dict(lam=1e4, mu=1.0, tau=1.0, alpha=1.0, inv_M=0.0)
    s_shift = 1e-2
    kL, kU = synthetic.lognormal_k(n, 1.0, 4)
    s = bmg.assemble(n, p["lam"], p["mu"], kfield(bmg, n, kL, kU), 1.0, p["tau"], p["alpha"], p["inv_M"])
    h = bmg.setup_hierarchy(s, "vanka", 1, 1, omega=0.7, n_coarse=8, p_shift=s_shift)
    H = mg.Hierarchy(n, fem.Params(**p), 1 / kL, 1 / kU, smoother="vanka", omega=0.7,
                     nu1=1, nu2=1, n_coarse=8, p_shift=s_shift)
    f = synthetic.rhs(n, 7)
    r = dev(bmg, n, f)
    z = torch.empty_like(r)
    h.vcycle(r, z)
    zo = H.vcycle(H.levels[0].mesh.pack(f))
    assert relmax(to_oracle(bmg, H.levels[0].mesh, z), zo) < 1e-9


def test_fp32_mg_solution_matches_oracle_direct_solve(bmg):
    """Mixed precision (FP32 V-cycle inside FP64 FGMRES): the solution against the oracle's
    direct sparse solve of the same system, element by element, n = 64, lambda = 1e4,
    lognormal K (sigma = 2)."""
    import scipy.sparse.linalg as spla
    import torch
    n = 64
    p = dict(lam=1e4, mu=1.0, tau=1.0, alpha=1.0, inv_M=1.0)
    kL, kU = synthetic.lognormal_k(n, 2.0, 11)
    s = bmg.assemble(n, p["lam"], p["mu"], kfield(bmg, n, kL, kU), 0.0, p["tau"], p["alpha"], p["inv_M"])
    h32 = bmg.setup_hierarchy(s, "vanka", 1, 1, omega=0.7, n_coarse=8, precision="fp32")
    f = synthetic.rhs(n, 1)
    b = dev(bmg, n, f)
    x = torch.zeros_like(b)
    info = h32.fgmres_solve(b, x, rtol=1e-8, maxit=400)
    assert info["status"] == "converged" and info["relres"] <= 1e-8
    m = Mesh(n)
    A = fem.assemble(m, fem.Params(**p), 1 / kL, 1 / kU)
    bo = m.pack(f)
    xo = np.zeros_like(bo)
    fi = m.free_idx
    xo[fi] = spla.spsolve(A[fi][:, fi].tocsc(), bo[fi])
    xg = to_oracle(bmg, m, x)
    assert np.linalg.norm(xg - xo) <= 1e-6 * np.linalg.norm(xo)
    assert relmax(xg, xo) <= 1e-5
    assert np.linalg.norm(bo - A @ xg) <= 1e-8 * np.linalg.norm(bo) * 1.0001


@pytest.mark.parametrize("smoother,omega", [("bsr", 0.7), ("vanka", 0.8)])
def test_fgmres_iterations_n128_match_oracle(bmg, smoother, omega):
    """FGMRES(50) counts at n = 128 (lambda = 1, K = 1, the sweep's first point): the GPU's
    FP64 solve against the oracle's.  Agreement here shows that the growth of the BSR counts
    with the grid is the inexact BSR's own, not a GPU defect that appears only at large n."""
    import torch
    n = 128
    p = dict(lam=1.0, mu=1.0, tau=1.0, alpha=1.0, inv_M=1.0)
    s = bmg.assemble(n, 1.0, 1.0, None, 1.0, 1.0, 1.0, 1.0)
    h = bmg.setup_hierarchy(s, smoother, 1, 1, omega=omega, omega_J=1.0, n_coarse=8)
    H = mg.Hierarchy(n, fem.Params(**p), np.ones((n, n)), np.ones((n, n)), smoother=smoother,
                     omega=omega, omega_J=1.0, n_coarse=8)
    f = synthetic.rhs(n, 0)
    b = dev(bmg, n, f)
    x = torch.zeros_like(b)
    info = h.fgmres_solve(b, x, rtol=1e-8, restart=50, maxit=400)
    A = H.levels[0].A
    _, oinfo = krylov.fgmres(A, H.levels[0].mesh.pack(f), H.vcycle, rtol=1e-8, restart=50, maxit=400)
    assert info["status"] == "converged" and oinfo["converged"]
    assert abs(info["iters"] - oinfo["iters"]) <= 1, (info["iters"], oinfo["iters"])


@pytest.mark.parametrize("smoother,omega", [("bsr", 0.7), ("vanka", 0.7)])
@pytest.mark.parametrize("n", [32, 64])
def test_w_cycle_parity(bmg, smoother, omega, n):
    """W(1,1) cycle (gamma = 2) against the oracle's, lognormal K, three and four levels."""
    import torch
    p = dict(lam=1e4, mu=1.0, tau=1.0, alpha=1.0, inv_M=1.0)
    kL, kU = synthetic.lognormal_k(n, 1.0, 12)
    s = bmg.assemble(n, p["lam"], p["mu"], kfield(bmg, n, kL, kU), 1.0, p["tau"], p["alpha"], p["inv_M"])
    h = bmg.setup_hierarchy(s, smoother, 1, 1, omega=omega, omega_J=1.0, n_coarse=8, cycle="W")
    H = mg.Hierarchy(n, fem.Params(**p), 1 / kL, 1 / kU, smoother=smoother, omega=omega,
                     omega_J=1.0, nu1=1, nu2=1, n_coarse=8, gamma=2)
    f = synthetic.rhs(n, 8)
    r = dev(bmg, n, f)
    z = torch.empty_like(r)
    h.vcycle(r, z)
    zo = H.vcycle(H.levels[0].mesh.pack(f))
    assert relmax(to_oracle(bmg, H.levels[0].mesh, z), zo) < 1e-9


def test_w_cycle_bsr_fgmres_iterations_match_oracle(bmg):
    """BSR with W(1,1) cycles, n = 64, unit parameters: FGMRES counts within one of the
    oracle's (and far below the V-cycle's, whose stationary iteration diverges here)."""
    import torch
    n = 64
    p = dict(lam=1.0, mu=1.0, tau=1.0, alpha=1.0, inv_M=1.0)
    s = bmg.assemble(n, 1.0, 1.0, None, 1.0, 1.0, 1.0, 1.0)
    hw = bmg.setup_hierarchy(s, "bsr", 1, 1, omega=0.7, omega_J=1.0, n_coarse=8, cycle="W")
    hv = bmg.setup_hierarchy(s, "bsr", 1, 1, omega=0.7, omega_J=1.0, n_coarse=8)
    H = mg.Hierarchy(n, fem.Params(**p), np.ones((n, n)), np.ones((n, n)), smoother="bsr",
                     omega=0.7, omega_J=1.0, n_coarse=8, gamma=2)
    f = synthetic.rhs(n, 0)
    b = dev(bmg, n, f)
    xw, xv = torch.zeros_like(b), torch.zeros_like(b)
    iw = hw.fgmres_solve(b, xw, rtol=1e-8, restart=50, maxit=400)
    iv = hv.fgmres_solve(b, xv, rtol=1e-8, restart=50, maxit=400)
    _, oinfo = krylov.fgmres(H.levels[0].A, H.levels[0].mesh.pack(f), H.vcycle, rtol=1e-8,
                             restart=50, maxit=400)
    assert iw["status"] == "converged" and oinfo["converged"]
    assert abs(iw["iters"] - oinfo["iters"]) <= 1, (iw["iters"], oinfo["iters"])
    assert iw["iters"] < iv["iters"]


@pytest.mark.parametrize("smoother,omega", [("vanka", 0.8), ("bsr", 0.7)])
@pytest.mark.parametrize("kind", ["const", "lognormal"])
def test_galerkin_vcycle_parity(bmg, smoother, omega, kind):
    """Galerkin coarse operators (coarse_op = GALERKIN, dense coarse elasticity element
    matrices) against the oracle's full sparse triple product P^T A P, n = 64 (four levels)."""
    import torch
    n = 64
    p = dict(lam=1e4, mu=1.0, tau=1.0, alpha=1.0, inv_M=1.0)
    if kind == "const":
        kL = kU = None
        kinvL = kinvU = np.ones((n, n))
    else:
        kL, kU = synthetic.lognormal_k(n, 1.0, 13)
        kinvL, kinvU = 1 / kL, 1 / kU
    Kf = None if kL is None else kfield(bmg, n, kL, kU)
    s = bmg.assemble(n, p["lam"], p["mu"], Kf, 1.0, p["tau"], p["alpha"], p["inv_M"])
    h = bmg.setup_hierarchy(s, smoother, 1, 1, omega=omega, omega_J=1.0, n_coarse=8, coarse_op="galerkin")
    H = mg.Hierarchy(n, fem.Params(**p), kinvL, kinvU, smoother=smoother, omega=omega, omega_J=1.0,
                     nu1=1, nu2=1, n_coarse=8, coarse_op="galerkin")
    f = synthetic.rhs(n, 9)
    r = dev(bmg, n, f)
    z = torch.empty_like(r)
    h.vcycle(r, z)
    zo = H.vcycle(H.levels[0].mesh.pack(f))
    assert relmax(to_oracle(bmg, H.levels[0].mesh, z), zo) < 1e-9


def test_galerkin_converges_where_rediscretisation_stagnates(bmg):
    """1/M = 1e-2 (the paper's (1/M) mu / alpha^2 group) with lambda = mu = K = 1: the
    two-grid LFA puts the rediscretised coarse-grid correction's spectral radius at 3.7 and
    V(1,1) Vanka's rho_LFA near 1 for every omega, while with Galerkin coarse operators it is
    0.82.  On the GPU the rediscretised FGMRES(50) makes no progress in 200 iterations; the
    Galerkin one converges, within one iteration of the oracle's count."""
    import torch
    n = 64
    p = dict(lam=1.0, mu=1.0, tau=1.0, alpha=1.0, inv_M=1e-2)
    s = bmg.assemble(n, 1.0, 1.0, None, 1.0, 1.0, 1.0, 1e-2)
    hr = bmg.setup_hierarchy(s, "vanka", 1, 1, omega=0.8, n_coarse=8)
    hg = bmg.setup_hierarchy(s, "vanka", 1, 1, omega=0.8, n_coarse=8, coarse_op="galerkin")
    f = synthetic.rhs(n, 0)
    b = dev(bmg, n, f)
    xr, xg = torch.zeros_like(b), torch.zeros_like(b)
    ir = hr.fgmres_solve(b, xr, rtol=1e-8, restart=50, maxit=200)
    ig = hg.fgmres_solve(b, xg, rtol=1e-8, restart=50, maxit=400)
    assert ir["status"] == "maxit" and ir["relres"] > 1e-3
    assert ig["status"] == "converged" and ig["relres"] <= 1e-8
    H = mg.Hierarchy(n, fem.Params(**p), np.ones((n, n)), np.ones((n, n)), smoother="vanka",
                     omega=0.8, n_coarse=8, coarse_op="galerkin")
    _, oinfo = krylov.fgmres(H.levels[0].A, H.levels[0].mesh.pack(f), H.vcycle, rtol=1e-8,
                             restart=50, maxit=400)
    assert oinfo["converged"] and abs(ig["iters"] - oinfo["iters"]) <= 1, (ig["iters"], oinfo["iters"])


@pytest.mark.parametrize("n", [8, 33])
def test_exact_divdiv_apply_parity(bmg, n):
    """bmg_assemble_divdiv(BMG_DIVDIV_EXACT): the original discretisation (Sec. 2.1, exact
    (div u, div v)) against the oracle's assembly with exact_divdiv, lognormal K, 1e-12."""
    import torch
    p = dict(lam=1e4, mu=1.3, tau=0.5, alpha=0.8, inv_M=1e-2)
    kL, kU = synthetic.lognormal_k(n, 1.5, 40 + n)
    s = bmg.assemble(n, p["lam"], p["mu"], kfield(bmg, n, kL, kU), 0.0, p["tau"], p["alpha"], p["inv_M"],
                     divdiv="exact")
    f = synthetic.uniform_field(n, 50 + n)
    x = dev(bmg, n, f)
    y = torch.empty_like(x)
    s.apply(x, y)
    m = Mesh(n)
    A = fem.assemble(m, fem.Params(exact_divdiv=True, **p), 1 / kL, 1 / kU)
    assert relmax(to_oracle(bmg, m, y), A @ m.pack(f)) < 1e-12


@pytest.mark.parametrize("smoother,omega", [("vanka", 0.7), ("bsr", 0.6)])
def test_exact_divdiv_vcycle_parity_and_degradation(bmg, smoother, omega):
    """V-cycle of the exact-div-div system against the oracle's (n = 32), and FGMRES counts
    at lambda / mu = 499 (nu = 0.499), K = 1e-6, n = 64: the exact form needs several times
    the reduced-quadrature form's iterations (the negative control of Table 1)."""
    import torch
    n = 32
    p = dict(lam=499.0, mu=1.0, tau=1.0, alpha=1.0, inv_M=1e-2)
    s = bmg.assemble(n, p["lam"], p["mu"], None, 1e-6, p["tau"], p["alpha"], p["inv_M"], divdiv="exact")
    h = bmg.setup_hierarchy(s, smoother, 1, 1, omega=omega, omega_J=1.0, n_coarse=8)
    kinv = np.full((n, n), 1e6)
    H = mg.Hierarchy(n, fem.Params(exact_divdiv=True, **p), kinv, kinv, smoother=smoother, omega=omega,
                     omega_J=1.0, nu1=1, nu2=1, n_coarse=8)
    f = synthetic.rhs(n, 10)
    r = dev(bmg, n, f)
    z = torch.empty_like(r)
    h.vcycle(r, z)
    zo = H.vcycle(H.levels[0].mesh.pack(f))
    assert relmax(to_oracle(bmg, H.levels[0].mesh, z), zo) < 1e-9
    n = 64
    its = {}
    for dd in ("reduced", "exact"):
        s = bmg.assemble(n, p["lam"], p["mu"], None, 1e-6, p["tau"], p["alpha"], p["inv_M"], divdiv=dd)
        h = bmg.setup_hierarchy(s, smoother, 1, 1, omega=omega, omega_J=1.0, n_coarse=8)
        b = dev(bmg, n, synthetic.rhs(n, 0))
        x = torch.zeros_like(b)
        its[dd] = h.fgmres_solve(b, x, rtol=1e-8, restart=50, maxit=1500)["iters"]
    assert its["exact"] >= 2 * its["reduced"], its


@pytest.mark.parametrize("kind", ["const", "lognormal"])
def test_fp32_vcycle_with_fp64_patch_solves(bmg, kind):
    """FP32 V-cycle whose Vanka patch solves use the FP64 inverses and FP64 products
    (patch_solve = BMG_PATCH_FP64): against the oracle's FP64 V-cycle within FP32 rounding
    (1e-5 relative, max-norm), n = 32; and an FGMRES solve with it meets 1e-8."""
    import torch
    n = 32
    p = dict(lam=1e4, mu=1.0, tau=1.0, alpha=1.0, inv_M=1.0)
    if kind == "const":
        kL = kU = None
        kinvL = kinvU = np.ones((n, n))
    else:
        kL, kU = synthetic.lognormal_k(n, 1.0, 14)
        kinvL, kinvU = 1 / kL, 1 / kU
    Kf = None if kL is None else kfield(bmg, n, kL, kU)
    s = bmg.assemble(n, p["lam"], p["mu"], Kf, 1.0, p["tau"], p["alpha"], p["inv_M"])
    h = bmg.setup_hierarchy(s, "vanka", 1, 1, omega=0.7, n_coarse=8, precision="fp32", patch_solve="fp64")
    H = mg.Hierarchy(n, fem.Params(**p), kinvL, kinvU, smoother="vanka", omega=0.7, nu1=1, nu2=1, n_coarse=8)
    f = synthetic.rhs(n, 15)
    r = dev(bmg, n, f)
    z = torch.empty_like(r)
    h.vcycle(r, z)
    zo = H.vcycle(H.levels[0].mesh.pack(f))
    assert relmax(to_oracle(bmg, H.levels[0].mesh, z), zo) < 1e-5
    x = torch.zeros_like(r)
    info = h.fgmres_solve(r, x, rtol=1e-8, maxit=400)
    assert info["status"] == "converged" and info["relres"] <= 1e-8


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_patch_thread_vanka_matches_row_tasks(bmg, precision):
    """The one-thread-per-patch Vanka solve (tiles 5-7) accumulates every output in the same
    order as the (row, patch) tasks (tiles 0-2), so the V-cycles agree to rounding (asserted:
    1e-6 relative in FP32, 1e-12 in FP64), n = 256, lognormal K (per-patch inverses)."""
    import torch
    n = 256
    kL, kU = synthetic.lognormal_k(n, 2.0, 11)
    s = bmg.assemble(n, 1e4, 1.0, kfield(bmg, n, kL, kU), 1.0, 1.0, 1.0, 1.0)
    r = dev(bmg, n, synthetic.rhs(n, 12))
    tol = 1e-6 if precision == "fp32" else 1e-12
    for a, b in ((0, 5), (1, 6), (2, 7)):
        z = []
        for tile in (a, b):
            h = setup_forced(bmg, s, "vanka", 0.7, tile, apply_tile=0, precision=precision)
            zz = torch.empty_like(r)
            h.vcycle(r, zz)
            z.append(zz.cpu().numpy())
            h.close()
        assert relmax(z[1], z[0]) <= tol, (a, b, relmax(z[1], z[0]))
