"""Damping parameters of the benchmark's V(1,1) cycles by two-grid LFA (Sec. 4.3 procedure).

For every parameter point of the 512 x 512 sweep (lambda in {1, 1e4, 1e6}, K in {1, 1e-6},
mu = tau = alpha = 1, 1/M in {1, 1e-2}) this script minimises rho_LFA (oracle/lfa.py) at
the sweep's fine grid, h = 1/512:
  * additive Vanka V(1,1): omega over [0.40, 1.20] in steps of 0.02;
  * inexact BSR V(1,1): (omega_J, omega) jointly, first on a 0.1 grid with 16 x 16 samples,
    then in steps of 0.02 around the best point with the paper's 32 x 32 samples (where
    rho_LFA does not depend on omega_J, the omega_J closest to 1 among the optima).
It writes tests/golden/omega_lfa.json (one record per point and smoother, with rho_LFA).
Test infrastructure: run by hand, ``python -m oracle.omega_table``; only oracle/ is called.
"""
from __future__ import annotations

import json
import os
import sys

import numpy as np

from . import fem, lfa

H = 1.0 / 512
LAMBDAS = (1.0, 1e4, 1e6)
KS = (1.0, 1e-6)
INV_MS = (1.0, 1e-2)


def vanka_point(prm, k):
    tg = lfa.TwoGrid(prm, k, H, "vanka")
    om, rho = lfa.optimise_omega(tg, 1, 1)
    return dict(omega=om, rho_lfa=round(rho, 4))


def bsr_point(prm, k):
    coarse = lfa.TwoGrid(prm, k, H, "bsr", samples=16)
    oj0, om0, _ = lfa.optimise_bsr(coarse, 1, 1, omegas=np.round(np.arange(0.4, 1.21, 0.1), 2),
                                   omegas_J=np.round(np.arange(0.6, 1.61, 0.1), 2), tie=1e-2)
    fine = lfa.TwoGrid(prm, k, H, "bsr")
    oms = np.round(np.arange(max(0.3, om0 - 0.1), om0 + 0.1001, 0.02), 2)
    ojs = np.round(np.arange(max(0.3, oj0 - 0.1), oj0 + 0.1001, 0.02), 2)
    oj, om, rho = lfa.optimise_bsr(fine, 1, 1, omegas=oms, omegas_J=ojs)
    return dict(omega_J=oj, omega=om, rho_lfa=round(rho, 4))


def main(path):
    out = []
    for inv_M in INV_MS:
        for lam in LAMBDAS:
            for k in KS:
                prm = fem.Params(lam=lam, mu=1.0, tau=1.0, alpha=1.0, inv_M=inv_M)
                rec = dict(lam=lam, K=k, inv_M=inv_M, h=H, nu1=1, nu2=1,
                           vanka=vanka_point(prm, k), bsr=bsr_point(prm, k))
                print(json.dumps(rec), flush=True)
                out.append(rec)
    with open(path, "w") as f:
        json.dump({"source": "two-grid LFA optimum of the V(1,1) cycle (Sec. 4.3: brute-force sampling "
                             "of omega in steps of 0.02; Sec. 4.1 Eq. real-TGM; App. C-D), written by "
                             "oracle/omega_table.py",
                   "points": out}, f, indent=1)


if __name__ == "__main__":
    main(sys.argv[1] if len(sys.argv) > 1 else
         os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "tests", "golden",
                      "omega_lfa.json"))
