"""The Galerkin coarse coefficients of the library (element.cpp, galerkin_coarsen_coefs),
compiled for the host: assembled over the coarse grids they give P^T A P of the oracle
(oracle/mg.py with coarse_op="galerkin", the full sparse triple product of Sec. 3's R = P^T)
on the displacement block, two levels down (32 -> 16 -> 8), to 1e-12 relative; and the
grad-div part is 4x its rediscretisation per level."""
import os
import shutil
import subprocess

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import fem, mg
from oracle.mesh import Mesh

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "..", "paper_2107_04060_gb300", "csrc")
INC = os.path.join(HERE, "..", "include")


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    out = tmp_path_factory.mktemp("gal") / "galerkin_host_check"
    cmd = [nvcc, "-std=c++17", "-O2", "-x", "c++", "-I", CSRC, "-I", INC,
           os.path.join(HERE, "galerkin_host_check.cpp"), os.path.join(CSRC, "element.cpp"),
           "-o", str(out)]
    subprocess.run(cmd, check=True, capture_output=True, timeout=300)
    return out


def assemble_u(m: Mesh, A, g, lam_area):
    rows, cols, vals = [], [], []
    for oi, o in enumerate(("L", "U")):
        E = np.asarray(A[oi]).reshape(9, 9) + lam_area * np.outer(g[oi], g[oi])
        for j in range(m.n):
            for i in range(m.n):
                d = m.tri_dofs(o, i, j)[:9]
                rows += list(np.repeat(d, 9))
                cols += list(np.tile(d, 9))
                vals += list(E.ravel())
    K = sp.coo_matrix((vals, (rows, cols)), shape=(m.ndof, m.ndof)).tocsr()
    keep = sp.diags(m.free.astype(float))
    return (keep @ K @ keep).tocsr()


@pytest.mark.parametrize("lam,mu", [(1.0, 1.0), (1e4, 1.3)])
def test_galerkin_coefficients_match_the_triple_product(checker, tmp_path, lam, mu):
    n, levels = 32, 2
    out = tmp_path / "coef.bin"
    subprocess.run([str(checker), str(n), str(levels), repr(lam), repr(mu), str(out)], check=True,
                   timeout=60)
    data = np.fromfile(out, dtype=np.float64).reshape(levels, 2 * 81 + 2 * 9 + 1)
    prm = fem.Params(lam=lam, mu=mu, tau=1.0, alpha=1.0, inv_M=1.0)
    H = mg.Hierarchy(n, prm, np.ones((n, n)), np.ones((n, n)), smoother="vanka", n_coarse=n >> levels,
                     coarse_op="galerkin")
    for l in range(1, levels + 1):
        A = data[l - 1, :162].reshape(2, 81)
        g = data[l - 1, 162:180].reshape(2, 9)
        lam_area = data[l - 1, 180]
        m = H.levels[l].mesh
        u = fem.type_mask(m, fem.U_TYPES).astype(float)
        du = sp.diags(u)
        want = (du @ H.levels[l].A @ du).tocsr()
        got = assemble_u(m, A, g, lam_area)
        scale = abs(want).max()
        assert abs(got - want).max() <= 1e-12 * scale
        # grad-div: lambda / |T| keeps the finest level's value, i.e. 4^l times the
        # rediscretised lambda / |T_l| of level l
        area_l = 0.5 / (m.n * m.n)
        assert lam_area == pytest.approx(lam / (0.5 / (n * n)), rel=1e-15)
        assert lam_area == pytest.approx(4 ** l * lam / area_l, rel=1e-15)
