"""Batched FGMRES (bmg_batch_create / bmg_batch_solve) against the single-instance solve and
the oracle's direct solve.

The batch runs, per instance, the same FGMRES(m) + V-cycle iteration as bmg_fgmres_solve
(Sec. 5.1); only the chunking of the dot-product reductions differs, so iteration counts
agree within one (three at lambda / mu = 1e6, where rounding alone moves the count of the
single solve by as much) and both solutions meet the 1e-8 relative residual, which bounds
their difference by about cond(A) * 1e-8 in the relative error measured below."""
import numpy as np
import pytest

import synthetic

pytestmark = pytest.mark.gpu

RTOL = 1e-8


def _problem(bmg, torch, n, lam, seed, sigma=1.0, omega=None):
    kL, kU = synthetic.lognormal_k(n, sigma, seed)
    K = torch.from_numpy(bmg.pack_k(n, kL, kU)).cuda()
    s = bmg.assemble(n, lam, 1.0, K, 1.0, 1.0, 1.0, 1.0)
    om = omega if omega is not None else (0.8 if lam < 10 else 0.7)
    h = bmg.setup_hierarchy(s, "vanka", 1, 1, omega=om)
    b = torch.from_numpy(bmg.pack(n, synthetic.rhs(n, 100 + seed))).cuda()
    return s, h, b


def _true_relres(s, b, x, torch):
    r = torch.empty_like(b)
    s.residual(b, x, r)
    return (torch.linalg.norm(r) / torch.linalg.norm(b)).item()


@pytest.fixture(scope="module")
def mixed():
    import torch
    import paper_2107_04060_gb300 as bmg
    torch.cuda.set_device(0)
    specs = [(16, 1.0), (32, 1e4), (64, 1e6), (32, 30.0), (16, 1e6), (64, 1.0), (8, 10.0)]
    probs = [_problem(bmg, torch, n, lam, q) for q, (n, lam) in enumerate(specs)]
    return bmg, torch, specs, probs


def test_batch_matches_single_solves(mixed):
    bmg, torch, specs, probs = mixed
    bt = bmg.Batch([p[1] for p in probs], rtol=RTOL, restart=50, maxit=400)
    xs = [torch.full_like(p[2], 7.0) for p in probs]      # x0_is_zero ignores the contents
    infos = bt.solve([p[2] for p in probs], xs)
    torch.cuda.synchronize()
    for (n, lam), (s, h, b), x, inf in zip(specs, probs, xs, infos):
        xr = torch.zeros_like(b)
        ir = h.fgmres_solve(b, xr, rtol=RTOL, restart=50, maxit=400)
        assert inf["status"] == "converged", (n, lam, inf)
        assert abs(inf["iters"] - ir["iters"]) <= (3 if lam >= 1e6 else 1), (n, lam, inf, ir)
        assert inf["relres"] <= RTOL
        assert _true_relres(s, b, x, torch) <= 1.01 * RTOL
        rel = (torch.linalg.norm(x - xr) / torch.linalg.norm(xr)).item()
        assert rel <= 1e-5, (n, lam, rel)
    assert bt.trips == max(i["iters"] for i in infos) + 1
    bt.close()


def test_batch_matches_oracle_direct_solve(mixed):
    from oracle import fem
    from oracle.adjoint import direct_solve
    from oracle.mesh import Mesh
    bmg, torch, specs, probs = mixed
    sel = [q for q, (n, _) in enumerate(specs) if n <= 16]
    bt = bmg.Batch([probs[q][1] for q in sel], rtol=1e-10, restart=50, maxit=400)
    xs = [torch.zeros_like(probs[q][2]) for q in sel]
    bt.solve([probs[q][2] for q in sel], xs)
    for q, x in zip(sel, xs):
        n, lam = specs[q]
        m = Mesh(n)
        kL, kU = synthetic.lognormal_k(n, 1.0, q)
        A = fem.assemble(m, fem.Params(lam=lam, mu=1.0, tau=1.0, alpha=1.0, inv_M=1.0), 1 / kL, 1 / kU)
        bo = m.pack(synthetic.rhs(n, 100 + q))
        xo = direct_solve(A, m, bo)
        xg = m.pack(bmg.unpack(n, x.cpu().numpy()))        # library layout -> oracle numbering
        fi = m.free_idx
        err = np.linalg.norm(xg[fi] - xo[fi]) / np.linalg.norm(xo[fi])
        assert err <= 1e-6, (n, lam, err)
    bt.close()


def test_batch_reuse_and_tiles_do_not_change_results(mixed):
    bmg, torch, specs, probs = mixed
    hs = [p[1] for p in probs]
    tuned = bmg.Batch(hs, rtol=RTOL, restart=20, maxit=400, autotune=True)
    for q, (n, _) in enumerate(specs):
        if n > 8:
            assert 0 <= tuned.tile("apply", n) < 5
            assert 0 <= tuned.tile("vanka", n) < 6
    bs = [p[2] for p in probs]
    x1 = [torch.zeros_like(b) for b in bs]
    i1 = tuned.solve(bs, x1)
    tuned.close()
    plain = bmg.Batch(hs, rtol=RTOL, restart=20, maxit=400, autotune=False)
    bs2 = [b.clone() for b in bs]                                  # same values, new buffers
    for _ in range(2):                                             # the graph is reused
        x2 = [torch.zeros_like(b) for b in bs2]
        i2 = plain.solve(bs2, x2)
        for a, c, ia, ic in zip(x1, x2, i1, i2):
            assert ia["iters"] == ic["iters"]
            assert torch.allclose(a, c, rtol=1e-12, atol=1e-14 * torch.abs(a).max().item())
    plain.close()


def test_batch_edge_cases(mixed):
    bmg, torch, specs, probs = mixed
    hs = [p[1] for p in probs[:3]]
    bs = [p[2].clone() for p in probs[:3]]
    bs[1].zero_()                                     # zero right-hand side: x = 0 at once
    bt = bmg.Batch(hs, rtol=RTOL, restart=50, maxit=400)
    xs = [torch.full_like(b, 3.0) for b in bs]
    infos = bt.solve(bs, xs)
    assert infos[1]["status"] == "converged" and infos[1]["iters"] == 0
    assert torch.count_nonzero(xs[1]).item() == 0
    assert infos[0]["status"] == "converged" and infos[2]["status"] == "converged"
    bt.close()
    # maxit = 0: one true residual, no Arnoldi step
    bt = bmg.Batch(hs, rtol=RTOL, restart=50, maxit=0)
    infos = bt.solve([p[2] for p in probs[:3]], [torch.zeros_like(b) for b in bs])
    assert all(i["status"] == "maxit" and i["iters"] == 0 and i["relres"] == pytest.approx(1.0)
               for i in infos)
    bt.close()
    # a non-finite right-hand side fails that instance only
    bt = bmg.Batch(hs, rtol=RTOL, restart=50, maxit=400)
    bad = [p[2].clone() for p in probs[:3]]
    bad[0][5] = float("nan")
    xs = [torch.zeros_like(b) for b in bad]
    with pytest.raises(bmg.BmgError, match="not finite"):
        bt.solve(bad, xs)
    assert _true_relres(probs[1][0], bad[1], xs[1], torch) <= 1.01 * RTOL
    bt.close()


def test_batch_rejects_invalid_batches(mixed):
    bmg, torch, specs, probs = mixed
    h0 = probs[0][1]
    with pytest.raises(bmg.BmgError, match="appears twice"):
        bmg.Batch([h0, h0])
    s, _, _ = _problem(bmg, torch, 16, 1.0, 0)
    hb = bmg.setup_hierarchy(s, "bsr", 1, 1, omega=0.7)
    with pytest.raises(bmg.BmgError, match="Vanka smoother in FP64"):
        bmg.Batch([h0, hb])
    h2 = bmg.setup_hierarchy(s, "vanka", 2, 2, omega=0.8)
    with pytest.raises(bmg.BmgError, match="share"):
        bmg.Batch([h0, h2])
    with pytest.raises(bmg.BmgError, match="restart"):
        bmg.Batch([h0], restart=0)


def test_batch_of_the_batched_workload_shape():
    """Instances of the batched workload's sizes {32, 64, 128, 256}, lambda log-uniform in
    [1, 1e6], lognormal K (sigma 1): every instance converges and meets the true residual."""
    import torch
    import paper_2107_04060_gb300 as bmg
    torch.cuda.set_device(0)
    rng = np.random.default_rng(7)
    probs, specs = [], []
    for q in range(8):
        n = int(rng.choice([32, 64, 128, 256]))
        lam = float(10 ** rng.uniform(0, 6))
        specs.append((n, lam))
        probs.append(_problem(bmg, torch, n, lam, 50 + q))
    bt = bmg.Batch([p[1] for p in probs], rtol=RTOL, restart=50, maxit=1000)
    xs = [torch.zeros_like(p[2]) for p in probs]
    infos = bt.solve([p[2] for p in probs], xs)
    for (n, lam), (s, h, b), x, inf in zip(specs, probs, xs, infos):
        assert inf["status"] == "converged", (n, lam, inf)
        assert _true_relres(s, b, x, torch) <= 1.01 * RTOL
    bt.close()
