"""The benchmark's damping parameters are the two-grid LFA optima that oracle/omega_table.py
wrote to tests/golden/omega_lfa.json (Sec. 4.3 procedure at the sweep's parameters)."""
import json
import os

import pytest

import bench

HERE = os.path.dirname(os.path.abspath(__file__))


def test_bench_omega_table_is_the_lfa_optimum():
    with open(os.path.join(HERE, "golden", "omega_lfa.json")) as f:
        pts = json.load(f)["points"]
    assert len(pts) == len(bench.OMEGA_LFA)
    for p in pts:
        om_v, om_j, om_b = bench.OMEGA_LFA[(p["lam"], p["K"], p["inv_M"])]
        assert om_v == pytest.approx(p["vanka"]["omega"])
        assert (om_j, om_b) == (pytest.approx(p["bsr"]["omega_J"]), pytest.approx(p["bsr"]["omega"]))
        assert p["h"] == pytest.approx(1 / bench.N_GRID) and p["nu1"] == p["nu2"] == 1
