"""The allocation-free FGMRES entry point (bmg_fgmres_solve_noalloc), for callers that cannot
allocate device memory while they run (a fixed memory budget, a framework that owns every
device allocation, or a context where cudaMalloc is not allowed).  It must give the same
solve as bmg_fgmres_solve, on two calls in a row (the second reuses the workspace the first
left behind), and refuse requests larger than its fixed workspace.

This file is collected last on purpose: if it fails, a run stopped at the first failure
has already run every other test.  It also passes alone in a fresh process (the first call
on the device sets up the workspace address)."""
import numpy as np
import pytest

import synthetic

pytestmark = pytest.mark.gpu


def test_noalloc_solve_matches_allocating_solve_twice():
    import torch
    import paper_2107_04060_gb300 as bmg
    torch.cuda.set_device(0)
    n = 32
    s = bmg.assemble(n, 1e4, 1.0, None, 1.0, 1.0, 1.0, 1.0)
    h = bmg.setup_hierarchy(s, "vanka", 1, 1, omega=0.7)
    for seed in (0, 3):                               # two calls in a row
        b = torch.from_numpy(bmg.pack(n, synthetic.rhs(n, seed))).cuda()
        x_ref = torch.zeros_like(b)
        x_na = torch.full_like(b, 5.0)                # garbage in: x0_is_zero ignores it
        i_ref = h.fgmres_solve(b, x_ref, rtol=1e-8, restart=30, maxit=400)
        i_na = h.fgmres_solve_noalloc(b, x_na, rtol=1e-8, restart=30, maxit=400)
        torch.cuda.synchronize()
        assert i_ref["status"] == "converged" and i_na["status"] == "converged"
        assert i_na["relres"] <= 1e-8
        assert abs(i_na["iters"] - i_ref["iters"]) <= 1
        rel = (torch.linalg.norm(x_na - x_ref) / torch.linalg.norm(x_ref)).item()
        assert rel <= 1e-6, rel


def test_noalloc_rejects_requests_beyond_the_workspace():
    import torch
    import paper_2107_04060_gb300 as bmg
    torch.cuda.set_device(0)
    n = 64                                            # allows restart <= 9
    s = bmg.assemble(n, 1.0, 1.0, None, 1.0, 1.0, 1.0, 1.0)
    h = bmg.setup_hierarchy(s, "vanka", 1, 1, omega=0.8)
    b = torch.from_numpy(bmg.pack(n, synthetic.rhs(n, 0))).cuda()
    x = torch.zeros_like(b)
    with pytest.raises(bmg.BmgError, match="exceed the fixed workspace"):
        h.fgmres_solve_noalloc(b, x, restart=30)
    assert bmg.noalloc_capacity() == 1 << 20
    info = h.fgmres_solve_noalloc(b, x, restart=9, maxit=400)
    assert info["status"] == "converged" and info["relres"] <= 1e-8
