"""The stored full-size oracle record (tests/golden/ot_n200000_oracle.json,
written by make_ot_n200000_oracle.py from the oracle alone) still matches the
workload generator and the oracle's sampling stream: its parameters are the
workload's, and its sampled rows' counts are re-derived here row by row (the
balanced-OT decision does not depend on the cost divisor, so the n*m divisor
sweep is not needed for them)."""
import json
import math
import os

import numpy as np

from paper_2306_06581_gb300 import inputs

HERE = os.path.dirname(os.path.abspath(__file__))


def test_stored_record_matches_workload_and_stream(orc):
    g = json.load(open(os.path.join(HERE, "golden", "ot_n200000_oracle.json")))
    w = inputs.ot_n200000()
    assert g["workload"] == w.name and (g["n"], g["m"], g["d"]) == (w.n, w.m, w.d)
    assert g["eps"] == w.eps and g["tol"] == w.tol and math.isclose(g["s"], w.s, rel_tol=1e-15)
    assert (g["seed"], g["pid"]) == (w.seed, w.pid) and g["status"] == 0
    # nnz of the whole sketch is within a few standard deviations of s (Eq. pois: E nnz = s without clipping)
    assert abs(g["nnz"] - w.s) < 6 * math.sqrt(w.s)
    f = lambda z: np.asarray(z, np.float32).astype(np.float64)
    P = orc.OracleProblem(f(w.a), f(w.b), w.eps, w.s, math.inf, x=f(w.x), y=f(w.y), seed=w.seed, pid=w.pid,
                          cost_norm=0)
    for i, cnt in g["row_nnz"].items():
        assert P.sample_row(int(i))["cols"].size == cnt, i
    t = g["terms"]
    assert abs(t["mass"] - 1.0) < 1e-6 and t["transport"] > 0


def test_stored_n1000000_record_matches_workload_and_stream(orc):
    """The 1,000,000-point record (make_ot_n1000000_oracle.py, skip sampler):
    parameters of the workload, sampled row counts re-derived row by row with
    the oracle's skip sampler, and the objective equal to its stored terms
    (OT: <T, C> - eps H(T); the sparse problem adds eps sum T log p*)."""
    g = json.load(open(os.path.join(HERE, "golden", "ot_n1000000_oracle.json")))
    w = inputs.ot_n1000000()
    assert g["workload"] == w.name and (g["n"], g["m"], g["d"]) == (w.n, w.m, w.d)
    assert g["eps"] == w.eps and g["tol"] == w.tol and math.isclose(g["s"], w.s, rel_tol=1e-15)
    assert (g["seed"], g["pid"], g["sampler"]) == (w.seed, w.pid, "skip") and g["status"] == 0
    assert abs(g["nnz"] - w.s) < 6 * math.sqrt(w.s)
    f = lambda z: np.asarray(z, np.float32).astype(np.float64)
    P = orc.OracleProblem(f(w.a), f(w.b), w.eps, w.s, math.inf, x=f(w.x), y=f(w.y), seed=w.seed, pid=w.pid,
                          cost_norm=0)
    for i, cnt in g["row_nnz"].items():
        assert P.skip_row(int(i))["cols"].size == cnt, i
    t = g["terms"]
    assert math.isclose(g["obj"], t["transport"] + w.eps * t["neg_entropy"], rel_tol=1e-12, abs_tol=1e-15)
    assert math.isclose(g["obj_sparse"], g["obj"] + w.eps * t["logp"], rel_tol=1e-12, abs_tol=1e-15)
    assert abs(t["mass"] - 1.0) < 1e-6 and t["transport"] > 0 and g["residual"] <= w.tol
