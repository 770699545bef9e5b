"""The FP32 operator variant whose input is staged in shared memory by TMA bulk tensor
copies (tile index 5) computes exactly what the same 32 x 8 tile computes from global
memory: the V-cycle outputs of two FP32 hierarchies, one forced to each variant, are equal
bit for bit (uniform K: the fine level reads K^{-1}; lognormal K: the coarse levels read
per-triangle 3 x 3 RT0 masses)."""
import os

import pytest

import synthetic

pytestmark = pytest.mark.gpu


def _hierarchy(bmg, torch, n, K, tile):
    os.environ["BMG_FORCE_APPLY_TILE"] = str(tile)
    try:
        if K is None:
            s = bmg.assemble(n, 1e4, 1.0, None, 1.0, 1.0, 1.0, 1.0)
        else:
            s = bmg.assemble(n, 1e4, 1.0, K, 0.0, 1.0, 1.0, 1.0)
        h = bmg.setup_hierarchy(s, "vanka", 1, 1, omega=0.7, precision="fp32")
    finally:
        del os.environ["BMG_FORCE_APPLY_TILE"]
    return s, h


@pytest.mark.parametrize("lognormal", [False, True])
def test_tma_operator_matches_global_loads_bitwise(lognormal):
    import torch
    import paper_2107_04060_gb300 as bmg
    torch.cuda.set_device(0)
    n = 256
    K = None
    if lognormal:
        kL, kU = synthetic.lognormal_k(n, 2.0, 4)
        K = torch.from_numpy(bmg.pack_k(n, kL, kU)).cuda()
    s5, h5 = _hierarchy(bmg, torch, n, K, 5)
    s0, h0 = _hierarchy(bmg, torch, n, K, 0)
    assert h5.tile(0, "apply") == 5 and h0.tile(0, "apply") == 0
    assert all(h5.tile(l, "apply") == 5 for l in range(h5.levels - 1) if (n >> l) >= 32)
    r = torch.from_numpy(bmg.pack(n, synthetic.rhs(n, 9))).cuda()
    z5, z0 = torch.empty_like(r), torch.empty_like(r)
    for _ in range(2):
        h5.vcycle(r, z5)
        h0.vcycle(r, z0)
        torch.cuda.synchronize()
        assert torch.equal(z5, z0)
        r = z0.clone()
    x5, x0 = torch.zeros_like(r), torch.zeros_like(r)
    b = torch.from_numpy(bmg.pack(n, synthetic.rhs(n, 10))).cuda()
    i5 = h5.fgmres_solve(b, x5, rtol=1e-8, maxit=300)
    i0 = h0.fgmres_solve(b, x0, rtol=1e-8, maxit=300)
    assert i5["status"] == "converged" and i5["iters"] == i0["iters"]
    assert torch.equal(x5, x0)


def test_bounded_tma_wait_reports_timeout_without_fault():
    """The wait of the TMA-staged FP32 operator on its bulk copies is bounded.  With the first
    wait's limit lowered to zero spins at setup (BMG_DEBUG_TMA_WAIT_LIMIT=0), every CTA gives
    up at once, records the timeout in the hierarchy's error flag, waits with the full limit
    for its own copies to land and returns: the solve reports BMG_ERR_CUDA with the reason,
    nothing faults, and the device stays usable."""
    import torch
    import paper_2107_04060_gb300 as bmg
    torch.cuda.set_device(0)
    n = 64
    os.environ["BMG_DEBUG_TMA_WAIT_LIMIT"] = "0"
    try:
        s, h = _hierarchy(bmg, torch, n, None, 5)
    finally:
        del os.environ["BMG_DEBUG_TMA_WAIT_LIMIT"]
    assert h.tile(0, "apply") == 5                     # the TMA variant is in use
    b = torch.from_numpy(bmg.pack(n, synthetic.rhs(n, 0))).cuda()
    x = torch.zeros_like(b)
    with pytest.raises(bmg.BmgError, match="CUDA error.*bulk-copy wait"):
        h.fgmres_solve(b, x, rtol=1e-8, maxit=3)
    torch.cuda.synchronize()                             # no sticky error: the context is fine
    s2, h2 = _hierarchy(bmg, torch, n, None, 5)
    x2 = torch.zeros_like(b)
    info = h2.fgmres_solve(b, x2, rtol=1e-8, maxit=300)
    assert info["status"] == "converged"
