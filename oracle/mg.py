"""Monolithic multigrid V-cycle (Sec. 3, Eq. TG-Operator-Biot; Sec. 5.1).

Levels n, n/2, ..., n_coarse (the paper: four levels, coarsest h = 1/8, direct solve).
Coarse operators are rediscretised (Sec. 3: "we use the rediscretization operators").  For a
per-triangle permeability the paper gives no coarse K; here the coarse RT0 mass is the
Galerkin product P_w^T M_w P_w, which is the exact rediscretisation with the fine-scale
K^{-1} (RT0 spaces are nested) and equals plain rediscretisation for constant K.

One V(nu1, nu2) cycle for A_l x = b_l from x = 0:
    nu1 relaxations; r = b - A x; x_c = V-cycle(R r) (or the direct solve on the coarsest
    level); x <- x + P x_c; nu2 relaxations.

W-cycles (gamma = 2): the coarse problem of each level approximated by two cycles, the
second on the residual the first leaves.  Galerkin coarse operators (coarse_op="galerkin"):
R A P on every level.

Pinned by: Table 2 / Table 3 two-grid factors and Table 4 iteration counts
(tests/test_oracle_mg.py); direct-solve parity through FGMRES (tests/test_oracle_mg.py); the
W-cycle by the two-grid factor and the LFA prediction it restores for multilevel inexact BSR;
Galerkin coarse operators by the nested-space identities (tests/test_oracle_mg.py,
tests/test_oracle_lfa.py).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import fem, transfer
from .mesh import Mesh
from .smoothers import Vanka, BraessSarazin


class Level:
    pass


class Hierarchy:
    """Operators, transfers and smoothers on every level."""

    def __init__(self, n: int, prm: fem.Params, kinv_L, kinv_U, smoother: str = "vanka",
                 omega: float = 0.8, omega_J: float = 1.0, nu1: int = 1, nu2: int = 1,
                 n_coarse: int = 8, coarse_op: str = "redisc", p_shift: float = 0.0,
                 w_essential: bool = False, gamma: int = 1, bsr_exact: bool = False):
        assert n >= n_coarse and (n // n_coarse) * n_coarse == n
        assert (n // n_coarse) & ((n // n_coarse) - 1) == 0, "n must be n_coarse * 2^k"
        self.prm = prm
        self.nu1, self.nu2 = nu1, nu2
        self.gamma = int(gamma)                 # coarse-grid cycles per level: 1 = V, 2 = W
        self.levels = []
        m = n
        while True:
            L = Level()
            L.mesh = Mesh(m, w_essential=w_essential)
            self.levels.append(L)
            if m == n_coarse:
                break
            m //= 2
        # operators
        f = self.levels[0]
        f.A = fem.assemble(f.mesh, prm, kinv_L, kinv_U)
        wmask_f = fem.type_mask(f.mesh, fem.W_TYPES)
        for lf, lc in zip(self.levels[:-1], self.levels[1:]):
            lf.P = transfer.prolongation(lf.mesh, lc.mesh)
            lf.R = transfer.restriction(lf.P)
            if coarse_op == "galerkin":
                lc.A = (lf.R @ lf.A @ lf.P).tocsr()
            else:
                zero = np.zeros((lc.mesh.n, lc.mesh.n))
                Ac = fem.assemble(lc.mesh, prm, zero, zero)           # all but the RT0 mass
                wf = fem.type_mask(lf.mesh, fem.W_TYPES)
                wc = fem.type_mask(lc.mesh, fem.W_TYPES)
                Mw_f = (sp.diags(wf.astype(float)) @ lf.A @ sp.diags(wf.astype(float)))
                Pw = (sp.diags(wf.astype(float)) @ lf.P @ sp.diags(wc.astype(float)))
                lc.A = (Ac + Pw.T @ Mw_f @ Pw).tocsr()
            lc.A.eliminate_zeros()
        del wmask_f
        # smoothers
        for L in self.levels[:-1]:
            if smoother == "vanka":
                L.smoother = Vanka(L.A, L.mesh, omega, p_shift=p_shift)
            elif smoother == "bsr":
                L.smoother = BraessSarazin(L.A, L.mesh, prm, omega, omega_J, exact=bsr_exact)
            else:
                raise ValueError(smoother)
        c = self.levels[-1]
        fi = c.mesh.free_idx
        c.free_idx = fi
        c.lu = spla.splu(c.A[fi][:, fi].tocsc())

    def coarse_solve(self, b: np.ndarray) -> np.ndarray:
        c = self.levels[-1]
        x = np.zeros_like(b)
        x[c.free_idx] = c.lu.solve(b[c.free_idx])
        return x

    def vcycle(self, b: np.ndarray, level: int = 0) -> np.ndarray:
        """Approximate A_level^{-1} b by one V(nu1, nu2) cycle from a zero initial guess
        (gamma = 2: a W-cycle, the coarse problem approximated by two cycles, the second on
        the residual left by the first; the coarsest level is solved directly either way)."""
        if level == len(self.levels) - 1:
            return self.coarse_solve(b)
        L = self.levels[level]
        x = np.zeros_like(b)
        for _ in range(self.nu1):
            x = L.smoother.sweep(L.A, b, x)
        r = b - L.A @ x
        rc = L.R @ r
        xc = self.vcycle(rc, level + 1)
        if level + 2 < len(self.levels):
            C = self.levels[level + 1]
            for _ in range(self.gamma - 1):
                xc = xc + self.vcycle(rc - C.A @ xc, level + 1)
        x = x + L.P @ xc
        for _ in range(self.nu2):
            x = L.smoother.sweep(L.A, b, x)
        return x


def two_grid_rho(h: Hierarchy, x0: np.ndarray, max_it: int = 200, tol: float = 1e-3,
                 min_it: int = 0):
    """Measured asymptotic factor rho_N = ||r_j|| / ||r_{j-1}|| of the stationary two-grid
    iteration with zero right-hand side (Sec. 4.3), stopped when consecutive factors differ
    by less than ``tol``.  The stopping test is applied from iteration ``min_it`` on: from a
    random start the factor rises slowly through a transient in which consecutive values can
    differ by less than 1e-3 long before the asymptotic value is reached.  ``h`` must have
    exactly two levels (exact coarse solve)."""
    assert len(h.levels) == 2
    L = h.levels[0]
    A = L.A
    b = np.zeros_like(x0)
    x = x0.copy()
    rn = np.linalg.norm(A @ x)
    rho_prev = None
    rhos = []
    for _ in range(max_it):
        for _ in range(h.nu1):
            x = L.smoother.sweep(A, b, x)
        r = b - A @ x
        x = x + L.P @ h.coarse_solve(L.R @ r)
        for _ in range(h.nu2):
            x = L.smoother.sweep(A, b, x)
        rn_new = np.linalg.norm(A @ x)
        rho = rn_new / rn
        rhos.append(rho)
        rn = rn_new
        if rho_prev is not None and len(rhos) >= min_it and abs(rho - rho_prev) < tol:
            break
        rho_prev = rho
        if rn == 0.0 or not np.isfinite(rn):
            break
    return rho, rhos
