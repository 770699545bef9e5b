"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module only draws random numbers and lays them out on the structured grid; it
holds none of the method's arithmetic.  Both the CPU oracle and the CUDA path take
their inputs from here, so that parity never depends on porting a random-number
generator.

Grid conventions (the triangulated unit square of the paper's Appendix A):
  * ``n`` cells per side, vertices ``(i, j)`` with ``0 <= i, j <= n`` (``i`` along x).
  * Cell ``(i, j)`` is cut along the diagonal from ``(i, j+1)`` to ``(i+1, j)`` into a
    lower-left triangle ``L`` and an upper-right triangle ``U``.
  * Edge families: ``h(i, j)`` from ``(i, j)`` to ``(i+1, j)``; ``v(i, j)`` from
    ``(i, j)`` to ``(i, j+1)``; ``d(i, j)`` the diagonal of cell ``(i, j)``.

Every field is a dict of 2-D arrays indexed ``[j, i]`` with these shapes:

  ux, uy   (n+1, n+1)   P1 displacement at vertices
  bh       (n+1, n)     bubble on h-edges        wh  (n+1, n)   RT0 on h-edges
  bv       (n, n+1)     bubble on v-edges        wv  (n, n+1)   RT0 on v-edges
  bd       (n, n)       bubble on d-edges        wd  (n, n)     RT0 on d-edges
  pL, pU   (n, n)       P0 pressure on the L / U triangle of each cell
"""
from __future__ import annotations

import numpy as np

TYPES = ("ux", "uy", "bh", "bv", "bd", "wh", "wv", "wd", "pL", "pU")


def shapes(n: int) -> dict:
    """Array shape ``(rows=j, cols=i)`` of every DoF type on an ``n``-cell grid."""
    return {
        "ux": (n + 1, n + 1), "uy": (n + 1, n + 1),
        "bh": (n + 1, n), "bv": (n, n + 1), "bd": (n, n),
        "wh": (n + 1, n), "wv": (n, n + 1), "wd": (n, n),
        "pL": (n, n), "pU": (n, n),
    }


def dirichlet_masks(n: int) -> dict:
    """Boolean masks of the displacement slots on the boundary (u = 0 there).

    Boundary-vertex P1 values and bubbles on boundary edges are constrained; RT0 and P0
    slots are all free (the pressure condition is natural in the mixed form).
    """
    m = {t: np.zeros(s, dtype=bool) for t, s in shapes(n).items()}
    for t in ("ux", "uy"):
        m[t][0, :] = m[t][-1, :] = True
        m[t][:, 0] = m[t][:, -1] = True
    m["bh"][0, :] = m["bh"][-1, :] = True     # h-edges on y = 0 and y = 1
    m["bv"][:, 0] = m["bv"][:, -1] = True     # v-edges on x = 0 and x = 1
    return m


def uniform_field(n: int, seed: int, lo: float = -1.0, hi: float = 1.0) -> dict:
    """Values uniform in [lo, hi] on every slot, drawn type by type in ``TYPES`` order
    from ``numpy.random.default_rng(seed)``; constrained displacement slots are zeroed."""
    rng = np.random.default_rng(seed)
    sh = shapes(n)
    out = {t: rng.uniform(lo, hi, size=sh[t]) for t in TYPES}
    for t, msk in dirichlet_masks(n).items():
        out[t][msk] = 0.0
    return out


def rhs(n: int, seed: int) -> dict:
    """Right-hand side uniform in [-1, 1] on the free DoFs (the workloads' recipe)."""
    return uniform_field(n, seed)


def lognormal_k(n: int, sigma: float, seed: int) -> tuple:
    """Per-triangle permeability ``K_T = exp(sigma * Z_T)``, ``Z_T ~ N(0, 1)``.

    Returns ``(K_L, K_U)``, each ``(n, n)`` indexed ``[j, i]``; the L array is drawn first.
    """
    rng = np.random.default_rng(seed)
    zl = rng.standard_normal((n, n))
    zu = rng.standard_normal((n, n))
    return np.exp(sigma * zl), np.exp(sigma * zu)


def constant_k(n: int, k: float) -> tuple:
    """Uniform permeability on every triangle."""
    return np.full((n, n), float(k)), np.full((n, n), float(k))
