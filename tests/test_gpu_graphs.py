"""V-cycles replayed from CUDA graphs (bmg_use_graphs) give exactly what the same cycle
launched kernel by kernel gives: bit for bit for a V-cycle, the same iterations and the same
solution for FGMRES, FP64 and FP32 hierarchies, with the Vanka and BSR smoothers and a
W-cycle.  The first cycle on a stream is launched kernel by kernel; the second captures the
graph for its (input, output) pair; later ones replay it."""
import pytest

import synthetic

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("smoother,precision,cycle", [("vanka", "fp64", "V"), ("bsr", "fp64", "V"),
                                                      ("vanka", "fp32", "V"), ("bsr", "fp64", "W")])
def test_graph_replay_matches_direct_launches(smoother, precision, cycle):
    import torch
    import paper_2107_04060_gb300 as bmg
    torch.cuda.set_device(0)
    n = 64
    s = bmg.assemble(n, 1e4, 1.0, None, 1.0, 1.0, 1.0, 1.0)
    h = bmg.setup_hierarchy(s, smoother, 1, 1, omega=0.7, precision=precision, cycle=cycle)
    b = torch.from_numpy(bmg.pack(n, synthetic.rhs(n, 3))).cuda()
    side = torch.cuda.Stream()
    prev = bmg.use_graphs(False)
    try:
        z_ref = torch.empty_like(b)
        h.vcycle(b, z_ref)                                # default stream, kernel by kernel
        torch.cuda.synchronize()
        bmg.use_graphs(True)
        zs = [torch.empty_like(b) for _ in range(4)]
        with torch.cuda.stream(side):
            for z in zs:                                  # direct, capture, replay, replay
                h.vcycle(b, z, stream=side)
        torch.cuda.synchronize()
        for z in zs:
            assert torch.equal(z, z_ref)
        # FGMRES with graphs against FGMRES without (same iterations, same solution)
        x1, x2 = torch.zeros_like(b), torch.zeros_like(b)
        i1 = h.fgmres_solve(b, x1, rtol=1e-8, maxit=400, stream=side)
        bmg.use_graphs(False)
        i2 = h.fgmres_solve(b, x2, rtol=1e-8, maxit=400, stream=side)
        torch.cuda.synchronize()
        assert i1["iters"] == i2["iters"] and i1["status"] == "converged"
        assert torch.equal(x1, x2)
    finally:
        bmg.use_graphs(prev)


def test_graph_replay_counts_its_kernels():
    import torch
    import paper_2107_04060_gb300 as bmg
    torch.cuda.set_device(0)
    n = 32
    s = bmg.assemble(n, 1.0, 1.0, None, 1.0, 1.0, 1.0, 1.0)
    h = bmg.setup_hierarchy(s, "vanka", 1, 1, omega=0.8)
    b = torch.from_numpy(bmg.pack(n, synthetic.rhs(n, 1))).cuda()
    z = torch.empty_like(b)
    side = torch.cuda.Stream()
    prev = bmg.use_graphs(True)
    try:
        with torch.cuda.stream(side):
            c0 = bmg.launch_count()
            h.vcycle(b, z, stream=side)                   # kernel by kernel
            c1 = bmg.launch_count()
            h.vcycle(b, z, stream=side)                   # captured and launched once
            c2 = bmg.launch_count()
            h.vcycle(b, z, stream=side)                   # replayed
            c3 = bmg.launch_count()
        torch.cuda.synchronize()
        assert c1 - c0 > 10 and c2 - c1 == c1 - c0 and c3 - c2 == c1 - c0
    finally:
        bmg.use_graphs(prev)
