"""Local Fourier analysis (LFA) of the two-grid method (Sec. 4; App. A-D).

Test infrastructure and an offline tool: it predicts the two-grid convergence factor
rho_LFA of Eq. real-TGM for additive Vanka (App. C) and inexact Braess-Sarazin (App. D)
relaxation, and chooses the damping parameters by brute-force sampling in steps of 0.02,
as Sec. 4.3 does.

Symbols.  Every operator of the two-grid cycle on the infinite uniform grid is block
Toeplitz over the 10 DoF types of a cell (Sec. 4.2: ux, uy, the three bubbles, the three RT0
fluxes, pL, pU).  A DoF of type t is placed at its cell index (i, j) (vertices, edges and
triangles are all indexed by the cell they belong to), so an operator with entries
A[(t, 0), (s, d)] has the 10 x 10 symbol

    A~(theta)[t, s] = sum_d A[(t, 0), (s, d)] exp(i theta . d)

(placing DoFs at their geometric positions instead multiplies every symbol by the same
diagonal unitary factors, which leaves every spectrum below unchanged).  The entries are
read from the oracle's assembled matrices (fem.assemble) on a small patch of cells with
the cell size h of the analysed grid, from the rows of the centre cell, where no boundary
condition reaches.

  * Operator: A~(theta), fine grid h; coarse operator: the rediscretised stencil on 2h
    evaluated at 2 theta (Sec. 3: rediscretisation).
  * Restriction R = P^T (Eq. block_interp), P read column by column from
    transfer.prolongation: for the harmonic theta^a = theta + pi a,
        R~_a[s, t] = sum P[(t, i), (s, I)] exp(i theta^a . (i - 2 I)),
    and interpolation P~_a = R~_a^H / 4 (the coarse mode exp(i 2 theta . I) spreads over
    the four harmonics).  The 10 x 40 and 40 x 10 symbols of Sec. 4.1 are [R~_a] and [P~_a].
  * Additive Vanka (App. C): M^{-1} = sum_l V_l^T D_l (V_l A V_l^T)^{-1} V_l over the
    20-DoF vertex patches; with the patch DoFs a = (t_a, offset d_a) from the vertex,
        M~^{-1}(theta)[t, s] = sum_{a, b: t_a = t, t_b = s} D_a (A_l^{-1})_{ab}
                               exp(i theta . (d_b - d_a)),
    D the natural weights (number of patches holding the DoF); E_s = I - omega M~^{-1} A~.
  * Inexact BSR (App. D): with F = blockdiag(additive Vanka on A_u with the 8-DoF patches,
    tau D_w), B the p-rows of A, and J = omega_J diag(S)^{-1},
        S = (1/M + alpha^2 / (lambda + 2 mu / d)) M_p + tau B_w D_w^{-1} B_w^T   (d = 2),
    the relaxation solves [[F, B^T], [B, -C_2]] (dy, dp) = r, i.e.
        dp = J (B F^{-1} r_y - r_p),   dy = F^{-1} (r_y - B^T dp),
    whose symbol is [[F~i - F~i B~^T J B~ F~i, F~i B~^T J], [J B~ F~i, -J]].
  * Two-grid symbol (Sec. 4.1): E_TG(theta) = E_s^nu2 (I - P~ A~_2h(2 theta)^{-1} R~ A~) E_s^nu1
    with A~ and E_s block diagonal over the four harmonics; rho_LFA = the largest spectral
    radius over the low frequencies theta in [-pi/2, pi/2)^2, sampled at 32 x 32 evenly
    spaced points offset so that none is at the origin (Sec. 4.3).

Pinned by: the rho_LFA and omega_opt printed in Table 2 (Vanka V(2,2)) and Table 3 (inexact
BSR V(1,1)), the nested Galerkin identities of the RT0 and P0 blocks, and the projection
property of the Galerkin coarse-grid correction (tests/test_oracle_lfa.py).
"""
from __future__ import annotations

import numpy as np

from . import fem, transfer
from .mesh import Mesh, TYPES

NT = len(TYPES)                                   # 10 DoF types
U_IDX = [TYPES.index(t) for t in fem.U_TYPES]
W_IDX = [TYPES.index(t) for t in fem.W_TYPES]
P_IDX = [TYPES.index(t) for t in fem.P_TYPES]
Y_IDX = U_IDX + W_IDX
HARMONICS = ((0, 0), (1, 0), (0, 1), (1, 1))
N_PATCH = 8                                       # cells per side of the stencil patch
C = N_PATCH // 2                                  # centre cell / vertex of the patch


def low_frequencies(samples: int = 32) -> np.ndarray:
    """(samples^2, 2) evenly spaced points of [-pi/2, pi/2)^2, offset by half a step so
    that none is at the origin (Sec. 4.3)."""
    t = -np.pi / 2 + (np.arange(samples) + 0.5) * np.pi / samples
    a, b = np.meshgrid(t, t, indexing="ij")
    return np.stack([a.ravel(), b.ravel()], axis=1)


def _locate(mesh: Mesh):
    """type index, i, j of every global DoF of a mesh."""
    typ = np.empty(mesh.ndof, dtype=np.int64)
    ii = np.empty(mesh.ndof, dtype=np.int64)
    jj = np.empty(mesh.ndof, dtype=np.int64)
    for k, t in enumerate(TYPES):
        r, c = mesh.shapes[t]
        o = mesh.offsets[t]
        jv, iv = np.divmod(np.arange(r * c), c)
        typ[o:o + r * c] = k
        ii[o:o + r * c] = iv
        jj[o:o + r * c] = jv
    return typ, ii, jj


class Entries:
    """Sparse description (row type, column type, offset, value) of a translation-invariant
    operator; ``symbol(theta)`` evaluates its (rows x cols) symbol at many frequencies."""

    def __init__(self, rt, ct, di, dj, val, nrow=NT, ncol=NT):
        self.rt = np.asarray(rt, dtype=np.int64)
        self.ct = np.asarray(ct, dtype=np.int64)
        self.di = np.asarray(di, dtype=float)
        self.dj = np.asarray(dj, dtype=float)
        self.val = np.asarray(val, dtype=float)
        self.nrow, self.ncol = nrow, ncol

    def symbol(self, theta: np.ndarray) -> np.ndarray:
        ph = np.exp(1j * (np.outer(theta[:, 0], self.di) + np.outer(theta[:, 1], self.dj)))
        out = np.zeros((len(theta), self.nrow * self.ncol), dtype=complex)
        flat = self.rt * self.ncol + self.ct
        for k in range(len(self.val)):            # a few hundred entries
            out[:, flat[k]] += self.val[k] * ph[:, k]
        return out.reshape(len(theta), self.nrow, self.ncol)


def operator_entries(prm: fem.Params, kinv: float, h: float) -> Entries:
    """Interior stencil of the reduced-quadrature operator on a grid of spacing h, read from
    the rows of the centre cell of a small assembled patch."""
    m = Mesh(N_PATCH)
    kin = np.full((N_PATCH, N_PATCH), float(kinv))
    A = fem.assemble(m, prm, kin, kin, h=h).tocsr()
    typ, ii, jj = _locate(m)
    rt, ct, di, dj, val = [], [], [], [], []
    for t in TYPES:
        r = int(m.idx(t, C, C))
        lo, hi = A.indptr[r], A.indptr[r + 1]
        for c, v in zip(A.indices[lo:hi], A.data[lo:hi]):
            rt.append(TYPES.index(t))
            ct.append(typ[c])
            di.append(ii[c] - C)
            dj.append(jj[c] - C)
            val.append(v)
    return Entries(rt, ct, di, dj, val)


def restriction_entries() -> Entries:
    """Entries of R = P^T (rows: coarse types, columns: fine types, offsets i - 2 I), from
    the columns of the oracle's P at the centre coarse cell.  P is independent of h."""
    fine, coarse = Mesh(2 * N_PATCH), Mesh(N_PATCH)
    P = transfer.prolongation(fine, coarse).tocsc()
    typ, ii, jj = _locate(fine)
    rt, ct, di, dj, val = [], [], [], [], []
    for s in TYPES:
        col = int(coarse.idx(s, C, C))
        lo, hi = P.indptr[col], P.indptr[col + 1]
        for r, v in zip(P.indices[lo:hi], P.data[lo:hi]):
            rt.append(TYPES.index(s))
            ct.append(typ[r])
            di.append(ii[r] - 2 * C)
            dj.append(jj[r] - 2 * C)
            val.append(v)
    return Entries(rt, ct, di, dj, val)


def vanka_entries(prm: fem.Params, kinv: float, h: float, with_flow: bool = True) -> Entries:
    """Entries of the additive Vanka operator M^{-1} = sum_l V_l^T D_l A_l^{-1} V_l (App. C):
    the interior vertex patch (20 DoFs, or the 8 displacement DoFs with ``with_flow=False``,
    taken from the displacement block of A), its exact inverse and natural weights."""
    m = Mesh(N_PATCH)
    kin = np.full((N_PATCH, N_PATCH), float(kinv))
    A = fem.assemble(m, prm, kin, kin, h=h).tocsr()
    if not with_flow:
        du = fem.type_mask(m, fem.U_TYPES).astype(float)
        A = A.multiply(du[:, None]).multiply(du[None, :]).tocsr()
    typ, ii, jj = _locate(m)
    patch = m.vertex_patch(C, C, with_flow)
    Al = A[patch][:, patch].toarray()
    inv = np.linalg.inv(Al)
    count = np.zeros(m.ndof)
    for j in range(C - 3, C + 4):                 # every patch that can reach the centre's DoFs
        for i in range(C - 3, C + 4):
            count[m.vertex_patch(i, j, with_flow)] += 1.0
    w = 1.0 / count[patch]
    pt = typ[patch]
    pdi = ii[patch] - C
    pdj = jj[patch] - C
    nd = len(patch)
    a, b = np.meshgrid(np.arange(nd), np.arange(nd), indexing="ij")
    a, b = a.ravel(), b.ravel()
    return Entries(pt[a], pt[b], pdi[b] - pdi[a], pdj[b] - pdj[a], w[a] * inv[a, b])


class TwoGrid:
    """Two-grid LFA of the monolithic method for one parameter set (constant K = k I).

    ``smoother`` is "vanka" or "bsr"; ``coarse`` is "redisc" (the rediscretised coarse
    operator, Sec. 3) or "galerkin" (its symbol R~ A~ P~).  The damping-independent symbols
    are formed once at the sample frequencies; ``rho(omega, nu1, nu2, omega_J)`` evaluates
    rho_LFA."""

    def __init__(self, prm: fem.Params, k: float, h: float, smoother: str = "vanka",
                 samples: int = 32, coarse: str = "redisc"):
        self.prm = prm
        self.smoother = smoother
        self.theta = low_frequencies(samples)
        kinv = 1.0 / k
        Aop = operator_entries(prm, kinv, h)
        Ac = operator_entries(prm, kinv, 2.0 * h)
        Rop = restriction_entries()
        self.L = []                               # A~(theta^a), 4 x (N, 10, 10)
        self.R = []                               # R~_a, 4 x (N, 10, 10)
        for a in HARMONICS:
            th = self.theta + np.pi * np.asarray(a, dtype=float)
            self.L.append(Aop.symbol(th))
            self.R.append(Rop.symbol(th))
        self.AH = Ac.symbol(2.0 * self.theta)
        N = len(self.theta)
        Lb = np.zeros((N, 4 * NT, 4 * NT), dtype=complex)
        Rb = np.zeros((N, NT, 4 * NT), dtype=complex)
        for a in range(4):
            Lb[:, a * NT:(a + 1) * NT, a * NT:(a + 1) * NT] = self.L[a]
            Rb[:, :, a * NT:(a + 1) * NT] = self.R[a]
        Pb = np.conj(np.transpose(Rb, (0, 2, 1))) / 4.0
        self.Lb, self.Rb, self.Pb = Lb, Rb, Pb
        if coarse == "galerkin":
            self.AH = Rb @ Lb @ Pb
        elif coarse != "redisc":
            raise ValueError(coarse)
        self.cgc = np.eye(4 * NT)[None] - Pb @ np.linalg.solve(self.AH, Rb @ Lb)
        if smoother == "vanka":
            self._minv = [vanka_entries(prm, kinv, h).symbol(self.theta + np.pi * np.asarray(a, float))
                          for a in HARMONICS]
        elif smoother in ("bsr", "bsr_exact"):
            self._bsr_parts(prm, kinv, h)
        else:
            raise ValueError(smoother)

    # -- inexact Braess-Sarazin ----------------------------------------------------------
    def _bsr_parts(self, prm, kinv, h):
        vu = vanka_entries(prm, kinv, h, with_flow=False)
        self._fu = [vu.symbol(self.theta + np.pi * np.asarray(a, float)) for a in HARMONICS]
        # tau D_w: the diagonal stencil entry of each RT0 type; diag(S) per P0 type
        ops = operator_entries(prm, kinv, h)
        tauDw = {}
        for t, s, di, dj, v in zip(ops.rt, ops.ct, ops.di, ops.dj, ops.val):
            if t == s and t in W_IDX and di == 0 and dj == 0:
                tauDw[t] = v
        area = 0.5 * h * h
        c_fs = prm.inv_M + prm.alpha ** 2 / (prm.lam + 2.0 * prm.mu / 2.0)
        diagS = {p: c_fs * area for p in P_IDX}
        for t, s, v in zip(ops.rt, ops.ct, ops.val):
            if t in P_IDX and s in W_IDX:
                diagS[t] += v * v / tauDw[s]
        self._tauDw = np.array([tauDw[t] for t in W_IDX])
        self._diagS = np.array([diagS[p] for p in P_IDX])
        self._c_fs_area = c_fs * area

    def _bsr_minv(self, a: int, omega_J: float) -> np.ndarray:
        """(N, 10, 10) symbol of the inexact BSR operator M^{-1} at harmonic a (exact BSR when
        the TwoGrid was made with smoother "bsr_exact": J = S~^{-1} with the symbol
        S~ = c_fs |T| I + (tau B_w)~ (tau D_w)^{-1} (tau B_w)~^H)."""
        N = len(self.theta)
        L = self.L[a]
        nu, nw = len(U_IDX), len(W_IDX)
        Fi = np.zeros((N, nu + nw, nu + nw), dtype=complex)
        Fi[:, :nu, :nu] = self._fu[a][:, U_IDX][:, :, U_IDX]
        Fi[:, nu:, nu:] = np.diag(1.0 / self._tauDw)[None]
        B = L[:, P_IDX][:, :, Y_IDX]               # (N, 2, 8)
        BT = L[:, Y_IDX][:, :, P_IDX]              # (N, 8, 2)
        if self.smoother == "bsr_exact":
            Bw = L[:, P_IDX][:, :, W_IDX]
            S = self._c_fs_area * np.eye(len(P_IDX))[None] + Bw @ np.diag(1.0 / self._tauDw)[None] @ \
                np.conj(np.transpose(Bw, (0, 2, 1)))
            J = np.linalg.inv(S)
        else:
            J = np.diag(omega_J / self._diagS)[None]
        FiBT = Fi @ BT
        JBFi = J @ B @ Fi
        M = np.zeros((N, NT, NT), dtype=complex)
        y = np.asarray(Y_IDX)
        p = np.asarray(P_IDX)
        M[:, y[:, None], y[None, :]] = Fi - FiBT @ JBFi
        M[:, y[:, None], p[None, :]] = FiBT @ J
        M[:, p[:, None], y[None, :]] = JBFi
        M[:, p[:, None], p[None, :]] = -J
        return M

    # -- two-grid factor -------------------------------------------------------------------
    def smoother_symbol(self, omega: float, omega_J: float = 1.0) -> np.ndarray:
        """(N, 40, 40) block-diagonal E_s = I - omega M~^{-1} A~ over the four harmonics."""
        N = len(self.theta)
        S = np.zeros((N, 4 * NT, 4 * NT), dtype=complex)
        for a in range(4):
            Mi = self._minv[a] if self.smoother == "vanka" else self._bsr_minv(a, omega_J)  # bsr, bsr_exact
            S[:, a * NT:(a + 1) * NT, a * NT:(a + 1) * NT] = np.eye(NT)[None] - omega * (Mi @ self.L[a])
        return S

    def rho(self, omega: float, nu1: int = 1, nu2: int = 1, omega_J: float = 1.0) -> float:
        S = self.smoother_symbol(omega, omega_J)
        T = self.cgc
        for _ in range(nu1):
            T = T @ S
        for _ in range(nu2):
            T = S @ T
        ev = np.linalg.eigvals(T)
        return float(np.max(np.abs(ev)))


def optimise_omega(tg: TwoGrid, nu1: int, nu2: int, omegas=None, omega_J: float = 1.0):
    """Brute-force minimisation of rho_LFA over omega in steps of 0.02 (Sec. 4.3).
    Returns (omega_opt, rho_opt)."""
    if omegas is None:
        omegas = np.round(np.arange(0.40, 1.2001, 0.02), 2)
    best = (None, np.inf)
    for om in omegas:
        r = tg.rho(float(om), nu1, nu2, omega_J)
        if r < best[1]:
            best = (float(om), r)
    return best


def optimise_bsr(tg: TwoGrid, nu1: int = 1, nu2: int = 1, omegas=None, omegas_J=None,
                 tie: float = 1e-3):
    """Joint brute-force minimisation over (omega_J, omega) in steps of 0.02 (Sec. 4.3,
    Table 3).  Where rho_LFA is flat in omega_J (it is limited by a mode that the Schur
    step does not touch), every omega_J within ``tie`` of the minimum is optimal; of those
    the one closest to 1 (plain Jacobi) is returned.  Returns (omega_J, omega, rho)."""
    if omegas is None:
        omegas = np.round(np.arange(0.40, 1.2001, 0.02), 2)
    if omegas_J is None:
        omegas_J = np.round(np.arange(0.70, 1.5001, 0.02), 2)
    res = []
    for oj in omegas_J:
        for om in omegas:
            res.append((float(oj), float(om), tg.rho(float(om), nu1, nu2, float(oj))))
    rmin = min(r for _, _, r in res)
    cand = [t for t in res if t[2] <= rmin + tie]
    return min(cand, key=lambda t: (abs(t[0] - 1.0), t[2]))
