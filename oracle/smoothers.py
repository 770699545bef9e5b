"""Relaxation schemes of the monolithic multigrid method (Sec. 3.2).

Additive Vanka (Sec. 3.2.1): with residual r = b - A x, solve on every vertex patch l
    (V_l A V_l^T) xhat_l = V_l r,
then  x <- x + omega * sum_l V_l^T D_l xhat_l,  D_l the natural weights (the reciprocal of
the number of patches holding the DoF).  Patches sit at every vertex, boundary vertices
included, restricted to free DoFs; the weights count the actual memberships.  Patch
matrices are extracted from the assembled operator and inverted with dense LU (FP64).

Inexact Braess-Sarazin (Sec. 3.2.2, App. D) on the saddle-point form [[A, B^T], [B, -C]]
with y = (u, w):
    F = blockdiag(additive Vanka on A_u^RQ with the 8-DoF displacement patches (Fig. 3 left),
                  tau D_w),   D_w = diag(M_w)
    S = (1/M + alpha^2 / (lambda + 2 mu / d)) M_p + tau B_w D_w^{-1} B_w^T      (d = 2)
    z     = F^{-1} r_y
    dp    = omega_J diag(S)^{-1} (B z - r_p)          (one weighted-Jacobi sweep on Eq. bsr_p)
    dy    = F^{-1} (r_y - B^T dp)
    x    <- x + omega (dy, dp)
The inner Vanka is undamped with natural weights.

Exact Braess-Sarazin (Sec. 3.2.2, ``exact=True``): the same steps with Eq. bsr_p solved,
dp = S^{-1} (B z - r_p), by a sparse LU of S.

Pinned by: the measured two-grid factors of Tables 2 and 3 (tests/test_oracle_mg.py); the
patch regularisation for 1/M = 0 by the identity "shifted patches at 1/M = 0 equal the
unshifted patches at 1/M = s" (tests/test_oracle_mg.py); exact BSR by both block equations
of its correction with S written out from its definition, and through the LFA by the
paper's exact-BSR remarks (tests/test_oracle_mg.py, tests/test_oracle_lfa.py).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .fem import U_TYPES, W_TYPES, P_TYPES, type_mask
from .mesh import Mesh


class Vanka:
    """Additive Vanka relaxation on vertex patches."""

    def __init__(self, A: sp.csr_matrix, mesh: Mesh, omega: float, with_flow: bool = True,
                 p_shift: float = 0.0):
        """``with_flow=False`` gives the 8-DoF displacement patches (A must then be the
        displacement block in the global numbering).

        ``p_shift`` = s >= 0 regularises the patches when 1/M = 0 (Sec. 5.3: a small weight
        on the diagonal of the Vanka blocks).  Reading: the weight multiplies the pressure
        mass with the sign of the -(1/M) M_p block, i.e. -s |T| is added to every P0
        diagonal entry of every patch matrix.  With this reading the shifted patch matrices
        of a system with 1/M = 0 are exactly the unshifted patch matrices of the same
        system with 1/M = s (pinned in tests/test_oracle_mg.py)."""
        self.omega = float(omega)
        n = mesh.n
        patches = [mesh.vertex_patch(i, j, with_flow) for j in range(n + 1) for i in range(n + 1)]
        patches = [p for p in patches if p]
        count = np.zeros(mesh.ndof)
        for p in patches:
            count[p] += 1.0
        self.weight = np.where(count > 0, 1.0 / np.maximum(count, 1.0), 0.0)
        pmask = type_mask(mesh, P_TYPES)
        A = A.tocsr()
        # group patches by size; invert V_l A V_l^T for each
        groups = {}
        for p in patches:
            groups.setdefault(len(p), []).append(p)
        self.groups = []
        for s, plist in groups.items():
            idx = np.array(plist, dtype=np.int64)                     # (G, s)
            # V_l A V_l^T for every patch of this size: entries A[idx[g, a], idx[g, b]]
            rows = np.repeat(idx[:, :, None], s, axis=2)
            cols = np.repeat(idx[:, None, :], s, axis=1)
            mats = np.asarray(A[rows.ravel(), cols.ravel()]).reshape(len(plist), s, s)
            if p_shift != 0.0:
                area = 0.5 * mesh.h * mesh.h
                mats[:, np.arange(s), np.arange(s)] -= p_shift * area * pmask[idx]
            inv = np.linalg.inv(mats)
            self.groups.append((idx, inv))

    def correction(self, r: np.ndarray) -> np.ndarray:
        """sum_l V_l^T D_l (V_l A V_l^T)^{-1} V_l r  (undamped)."""
        out = np.zeros_like(r)
        for idx, inv in self.groups:
            xhat = np.einsum("gab,gb->ga", inv, r[idx])
            np.add.at(out, idx, xhat * self.weight[idx])
        return out

    def sweep(self, A: sp.csr_matrix, b: np.ndarray, x: np.ndarray) -> np.ndarray:
        """One relaxation step x <- x + omega M^{-1} (b - A x)."""
        r = b - A @ x
        return x + self.omega * self.correction(r)


class BraessSarazin:
    """Inexact Braess-Sarazin relaxation with the fixed-stress Schur approximation."""

    def __init__(self, A: sp.csr_matrix, mesh: Mesh, prm, omega: float, omega_J: float,
                 exact: bool = False):
        """``exact=True``: exact Braess-Sarazin (Sec. 3.2.2, Eq. bsr_p solved exactly): the
        pressure step solves S dp = B z - r_p with a sparse LU of S instead of one weighted
        Jacobi sweep (omega_J is then unused)."""
        self.omega = float(omega)
        self.omega_J = float(omega_J)
        self.exact = bool(exact)
        self.mu_ = type_mask(mesh, U_TYPES)
        self.mw_ = type_mask(mesh, W_TYPES)
        self.mp_ = type_mask(mesh, P_TYPES)
        A = A.tocsr()
        du = sp.diags(self.mu_.astype(float))
        dw = sp.diags(self.mw_.astype(float))
        dp = sp.diags(self.mp_.astype(float))
        Au = (du @ A @ du).tocsr()
        self.vanka_u = Vanka(Au, mesh, 1.0, with_flow=False)
        diagA = A.diagonal()
        self.tauDw = np.where(self.mw_ & mesh.free, diagA, 0.0)          # tau D_w
        self.Bu = (dp @ A @ du).tocsr()                                   # alpha B_u (p rows)
        self.Bw = (dp @ A @ dw).tocsr()                                   # tau B_w   (p rows)
        # diag(S): (1/M + alpha^2/(lambda + mu)) |T| + sum_e (tau B_w)_{T,e}^2 / (tau D_w)_e
        area = 0.5 * mesh.h * mesh.h
        d = 2.0
        c_fs = prm.inv_M + prm.alpha ** 2 / (prm.lam + 2.0 * prm.mu / d)
        inv_tauDw = np.where(self.tauDw != 0.0, 1.0 / np.where(self.tauDw != 0.0, self.tauDw, 1.0), 0.0)
        Bw2 = self.Bw.multiply(self.Bw).tocsr()
        self.diagS = np.where(self.mp_, c_fs * area, 0.0) + Bw2 @ inv_tauDw
        self.inv_tauDw = inv_tauDw
        if self.exact:
            # S = c_fs M_p + tau B_w D_w^{-1} B_w^T on the P0 DoFs
            pidx = np.nonzero(self.mp_)[0]
            S = (sp.diags(np.where(self.mp_, c_fs * area, 0.0)) +
                 self.Bw @ sp.diags(inv_tauDw) @ self.Bw.T).tocsr()[pidx][:, pidx]
            self.pidx = pidx
            self.S_lu = spla.splu(S.tocsc())

    def F_inv(self, ry: np.ndarray) -> np.ndarray:
        """F^{-1} applied to a vector whose u and w parts are used (p part ignored)."""
        z = self.vanka_u.correction(np.where(self.mu_, ry, 0.0))
        z = np.where(self.mu_, z, 0.0) + np.where(self.mw_, ry * self.inv_tauDw, 0.0)
        return z

    def correction(self, r: np.ndarray) -> np.ndarray:
        """The undamped BSR update (dy, dp) for residual r."""
        ry = np.where(self.mp_, 0.0, r)
        rp = np.where(self.mp_, r, 0.0)
        z = self.F_inv(ry)
        Bz = self.Bu @ z + self.Bw @ z
        if self.exact:
            dp = np.zeros_like(r)
            dp[self.pidx] = self.S_lu.solve((Bz - rp)[self.pidx])
        else:
            dp = np.where(self.mp_, self.omega_J * (Bz - rp) / np.where(self.diagS != 0, self.diagS, 1.0), 0.0)
        BTdp = self.Bu.T @ dp + self.Bw.T @ dp
        dy = self.F_inv(ry - BTdp)
        return dy + dp

    def sweep(self, A: sp.csr_matrix, b: np.ndarray, x: np.ndarray) -> np.ndarray:
        r = b - A @ x
        return x + self.omega * self.correction(r)
