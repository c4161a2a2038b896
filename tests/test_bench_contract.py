"""Host-side pieces of bench.py's JSON line (CPU): the DRAM traffic of the
roofline comes from the committed ncu summaries of the benchmarked workloads,
the algorithmic bytes follow the iteration's definition, and the workload
names line up with those summaries."""
import math
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_2306_06581_gb300 import inputs  # noqa: E402


@pytest.mark.parametrize("make,expect", [(inputs.uot_n20000, 1.6e6), (inputs.ot_n200000, 5.12e8)])
def test_traffic_from_committed_profiles(make, expect):
    w = make()
    assert bench._traffic(w.name) == pytest.approx(expect)
    src = open(os.path.join(ROOT, "profiles", f"spmv_traffic_{w.name}.txt")).read()
    ref = src.split("source:", 1)[1].split()[0]
    assert os.path.exists(os.path.join(ROOT, ref)), ref


def test_traffic_absent_is_null():
    assert bench._traffic("no_such_workload") is None


def test_spmv_bytes_definition():
    n, m, nnz = 20000, 20000, 3167743
    row, col = bench._spmv_bytes({"nnz": nnz}, n, m, "f32", 0)
    # every element once per pass (index + value), pointers, and the per-row / gathered vectors
    assert row == nnz * 8 + 4 * (n + 1) + 4 * n * 3 + 4 * m
    assert col == nnz * 8 + 4 * (m + 1) + 4 * m * 3 + 4 * n
    r2, c2 = bench._spmv_bytes({"nnz": nnz}, n, m, "bf16", 1)
    assert r2 < row and c2 < col   # two-byte values outweigh the extra stabilised vectors here
    assert math.isclose(row + col, 51483896, rel_tol=0)   # the figure the default line reports
