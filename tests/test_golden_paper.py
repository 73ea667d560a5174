"""Values printed in the paper (tests/golden/*, each file cites its passage)."""
import os

import numpy as np

import pamd_inputs as pi

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _read_numbers(name):
    rows = [l.split() for l in open(os.path.join(GOLD, name)) if l.strip() and not l.startswith("#")]
    return rows


def test_paper_temperature_set_is_geometric():
    temps = np.array([float(v) for v in _read_numbers("paper_temperatures.txt")[0]])
    sched = pi.geometric_schedule(temps[0], temps[-1], len(temps) - 1)
    assert np.all(np.abs(sched - temps) <= 0.6), (sched, temps)
    assert np.all(np.diff(temps) < 0)


def test_paper_budget_arithmetic():
    g = {k: float(v) for k, v, *_ in _read_numbers("paper_budget.txt")}
    fs_to_ns = 1e-6
    pa = g["replicas"] * g["theta_pa"] * g["temperatures"] * g["dt_fs"] * fs_to_ns
    assert abs(pa - g["pa_total_ns"]) < 1e-9
    pt = g["pt_exchanges"] * g["theta_pt"] * g["temperatures"] * g["dt_fs"] * fs_to_ns
    assert abs(pt - g["pt_production_ns"]) < 1e-9
    assert g["pt_production_ns"] + g["pt_equilibration_ns"] == g["total_budget_ns"]
    assert g["canonical_ns_per_temperature"] * g["temperatures"] == g["total_budget_ns"]
