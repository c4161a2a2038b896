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


@pytest.mark.parametrize("make,expect", [(inputs.uot_n20000, 1.6e6), (inputs.ot_n200000, 5.418e8),
                                         (inputs.ot_n1000000, 3.1486e9)])
def test_traffic_from_committed_profiles(make, expect):
    w = make()
    traffic, src_name = bench._traffic(w.name)
    assert traffic == pytest.approx(expect)
    assert src_name == f"profiles/spmv_traffic_{w.name}.txt"
    src = open(os.path.join(ROOT, src_name)).read()
    ref = src.split("source:", 1)[1].split()[0]
    assert os.path.exists(os.path.join(ROOT, ref)), ref


def test_traffic_absent_is_null():
    assert bench._traffic("no_such_workload") == (None, None)


def test_roofline_bound_label_follows_measured_traffic():
    # the 20000-point UOT sketch stays in L2: 1.6 MB of DRAM per iteration against 51.5 MB algorithmic
    assert bench._bound(1.6e6, 51483896) == "l2-effective"
    # the 200000-point sketch streams from DRAM: 512 MB measured against 479 MB algorithmic
    assert bench._bound(5.12e8, 479118184) == "hbm"
    assert bench._bound(None, 1.0).startswith("hbm (traffic not measured")


def test_dense_cap_is_automatic_only_for_large_problems():
    class A:
        dense_cap = 0
    assert bench._dense_cap(A(), bench._workload("ot_n1000000", 200000)) == 2
    assert bench._dense_cap(A(), bench._workload("uot_n20000")) == 20000
    A.dense_cap = 5
    assert bench._dense_cap(A(), bench._workload("uot_n20000")) == 5


def test_spmv_bytes_definition():
    n, m, nnz = 20000, 20000, 3167743
    row, col = bench._spmv_bytes({"nnz": nnz}, n, m, "f32", 0)
    # every element once per pass (index + value), pointers, and the per-row / gathered vectors
    assert row == nnz * 8 + 4 * (n + 1) + 4 * n * 3 + 4 * m
    assert col == nnz * 8 + 4 * (m + 1) + 4 * m * 3 + 4 * n
    r2, c2 = bench._spmv_bytes({"nnz": nnz}, n, m, "bf16", 1)
    assert r2 < row and c2 < col   # two-byte values outweigh the extra stabilised vectors here
    assert math.isclose(row + col, 51483896, rel_tol=0)   # the figure the default line reports


def test_workloads_and_their_modes():
    names = {"uot_n20000": (20000, 1.0, 0), "ot_n1000": (1000, math.inf, 0), "ot_n200000": (200000, math.inf, 1),
             "ot_n1000000": (1000000, math.inf, 1)}
    assert set(bench.WORKLOADS) == set(names) | {"frames64"}
    for name, (n, lam, logd) in names.items():
        w = bench._workload(name)
        assert w.n == n and w.lam == lam and bench._log_domain(w) == logd
        cfg = bench._config(w, "flushed")
        assert cfg["workload"] == w.name and cfg["n"] == n and cfg["log_domain"] == logd
        assert cfg["lambda"] == (None if math.isinf(lam) else lam)
    # --n re-draws the same family at another size
    assert bench._workload("uot_n20000", 2000).n == 2000
    with pytest.raises(SystemExit):
        bench._workload("no_such_workload")


def test_frames_batch_budgets():
    sets, pairs, s = bench._frames_batch()
    assert len(pairs) == 2016 and len(s) == 2016
    for (i, j), sp in zip(pairs[:50], s[:50]):
        nij = math.sqrt(len(sets[i][1]) * len(sets[j][1]))
        assert sp == pytest.approx(8.0 * 1e-3 * nij * math.log(nij) ** 4)


def test_peak_is_the_measured_copy_bandwidth():
    peak, kind = bench._peaks()
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        import json
        assert kind == "measured" and peak == json.load(open(path))["hbm_gbs"]
    else:
        assert (peak, kind) == (6800.0, "fallback")


def test_reference_arm_prints_one_contract_line():
    # the reference arm (the FP64 oracle on the host cores) end to end, on the small balanced workload
    import json
    import subprocess
    import sys
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
                        "ot_n1000", "--steps", "1", "--warmup", "0"], capture_output=True, text=True, timeout=600,
                       cwd=ROOT, env=dict(os.environ, RANK="0", WORLD_SIZE="1"))
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [l for l in p.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["higher_is_better"] is False and d["value"] > 0
    assert d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["config"]["workload"] == inputs.ot_n1000().name
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_kernel_time_excludes_the_iteration_setup():
    # 1 setup iteration (log domain) + 199 kernel iterations; 30 ms of the phase is setup
    r = {"ms_iter": 30.0 + 199 * 0.9, "ms_setup": 30.0, "iters_enqueued": 200}
    assert abs(bench._kernel_ms_per_iteration(r, 1) - 0.9) < 1e-12
    r = {"ms_iter": 0.01 + 200 * 0.2, "ms_setup": 0.01, "iters_enqueued": 200}
    assert abs(bench._kernel_ms_per_iteration(r, 0) - 0.2) < 1e-12


def test_stream_bytes_replace_the_element_bytes_only():
    res = {"nnz": 1000, "stream_bytes": 7000}
    row, col = bench._spmv_bytes(res, 100, 120, "f32", 1)
    vec = row + col - 2 * 1000 * 8 - 4 * 101 - 4 * 121
    assert bench._stream_bytes(res, 100, 120, "f32", 1) == 7000 + vec
    assert bench._stream_bytes({"nnz": 1000, "stream_bytes": 0}, 100, 120, "f32", 1) is None
