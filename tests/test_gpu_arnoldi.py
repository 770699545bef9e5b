"""The library's Arnoldi process (Sec. 5.1's FGMRES: classical Gram-Schmidt with one
re-orthogonalisation; first pass FP32, update FP64, second pass and final correction in
double-float arithmetic) against the same FGMRES(m) written here in plain PyTorch FP64 on
the same operator and V-cycle.

The nearly incompressible case (lambda = 1e6 on a 512^2 grid) is the sensitive one: there the
true residual of FP64 FGMRES lags its least-squares estimate by a few times 1e-8 (rounding of
the operator application, amplified by the operator's conditioning), so whether a solve to
1e-8 needs one more restart cycle depends on rounding details.  On two of six right-hand
sides the library needs about 80 iterations at rtol 1e-8 and 62 at rtol 1.1e-8, where the
FP64 reference needs 62.  The test therefore compares the true residual after fixed
iteration counts inside and at the end of the first restart cycle, and the converged
solution."""
import numpy as np
import pytest

import synthetic

pytestmark = pytest.mark.gpu


def fgmres_fp64(s, h, b, rtol, m, maxit):
    """Right-preconditioned FGMRES(m), CGS2 in FP64 (torch), Givens least squares (numpy)."""
    import torch
    x = torch.zeros_like(b)
    r = torch.empty_like(b)
    w = torch.empty_like(b)
    bn = torch.linalg.norm(b).item()
    its = 0
    while True:
        s.residual(b, x, r)
        beta = torch.linalg.norm(r).item()
        if beta <= rtol * bn or its >= maxit:
            return its, beta / bn, x
        V = torch.zeros(m + 1, b.numel(), dtype=b.dtype, device=b.device)
        Z = torch.zeros(m, b.numel(), dtype=b.dtype, device=b.device)
        H = np.zeros((m + 1, m))
        cs, sn, g = np.zeros(m), np.zeros(m), np.zeros(m + 1)
        g[0] = beta
        V[0] = r / beta
        k = 0
        for j in range(m):
            h.vcycle(V[j], Z[j])
            s.apply(Z[j], w)
            for _ in range(2):
                c = V[: j + 1] @ w
                w -= V[: j + 1].T @ c
                H[: j + 1, j] += c.cpu().numpy()
            H[j + 1, j] = torch.linalg.norm(w).item()
            V[j + 1] = w / H[j + 1, j]
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            den = np.hypot(H[j, j], H[j + 1, j])
            cs[j], sn[j] = H[j, j] / den, H[j + 1, j] / den
            H[j, j], H[j + 1, j] = den, 0.0
            g[j + 1], g[j] = -sn[j] * g[j], cs[j] * g[j]
            k = j + 1
            its += 1
            if abs(g[j + 1]) <= rtol * bn or its >= maxit:
                break
        y = np.zeros(k)
        for i in range(k - 1, -1, -1):
            y[i] = (g[i] - H[i, i + 1:k] @ y[i + 1:k]) / H[i, i]
        x += Z[:k].T @ torch.from_numpy(y).to(b.device)


@pytest.mark.parametrize("seed", [0, 3])
def test_arnoldi_matches_fp64_gram_schmidt_nearly_incompressible(seed):
    import torch
    import paper_2107_04060_gb300 as bmg
    torch.cuda.set_device(0)
    n = 512
    s = bmg.assemble(n, 1e6, 1.0, None, 1.0, 1.0, 1.0, 1.0)
    h = bmg.setup_hierarchy(s, "vanka", 1, 1, omega=0.7)
    b = torch.from_numpy(bmg.pack(n, synthetic.rhs(n, seed))).cuda()
    for maxit, tol in ((30, 1e-4), (50, 3e-2)):
        x = torch.zeros_like(b)
        info = h.fgmres_solve(b, x, rtol=1e-12, restart=50, maxit=maxit)
        its_ref, relres_ref, x_ref = fgmres_fp64(s, h, b, 1e-12, 50, maxit)
        assert info["iters"] == its_ref == maxit
        assert abs(info["relres"] / relres_ref - 1.0) <= tol, (maxit, info["relres"], relres_ref)
    x = torch.zeros_like(b)
    info = h.fgmres_solve(b, x, rtol=1e-8, restart=50, maxit=400)
    _, relres_ref, x_ref = fgmres_fp64(s, h, b, 1e-8, 50, 400)
    assert info["status"] == "converged" and relres_ref <= 1e-8
    r = torch.empty_like(b)
    s.residual(b, x, r)
    assert (torch.linalg.norm(r) / torch.linalg.norm(b)).item() <= 1.0001e-8
    rel = (torch.linalg.norm(x - x_ref) / torch.linalg.norm(x_ref)).item()
    assert rel <= 1e-4, rel
