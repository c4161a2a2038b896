"""Benchmark: Spar-Sink time to marginal error 1e-5 vs dense Sinkhorn on one GB300.

A step is one complete Spar-Sink solve of the workload (sketch construction,
scaling iterations until the stopping residual is <= 1e-5, objective), with
the inputs resident in HBM; L2 is flushed (a 512 MB write) between timed steps.
Default workload: UOT, lambda = 1, n = m = 20000 points in R^10 (3-component
Gaussian mixture vs multivariate t with 3 degrees of freedom), eps = 0.05,
s = 16 n ln n, FP32 values and iterates.

One JSON line on rank 0.  `value` is the time per solve (ms, lower is better);
under torchrun every rank solves its own replica (weak scaling, no data-path
collective) and the max over ranks is reported.  Extra keys: roofline of the
SpMV half-iterations, the dense Sinkhorn comparison on the same GPU, the CPU
oracle baseline, clocks sampled during the timed region, the end-to-end time
through the public API with host buffers, and the kernel launch count.

`--impl reference` times the FP64 CPU oracle (the only reference this method
has) on the same workload, metric and unit.
"""
from __future__ import annotations

import argparse
import csv
import io
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Spar-Sink time-to-marginal-err 1e-5 vs dense Sinkhorn on GB300; SpMV HBM GB/s"
UNIT = "ms"
TOL = 1e-5


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d.get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


def _workload(name):
    from paper_2306_06581_gb300 import inputs
    if name == "uot_n20000":
        return inputs.uot_n20000()
    if name == "ot_n1000":
        return inputs.ot_n1000()
    raise SystemExit(f"unknown workload {name}")


def _config(w, flush):
    return {"workload": w.name, "n": w.n, "m": w.m, "d": w.d, "eps": w.eps,
            "lambda": None if math.isinf(w.lam) else w.lam, "s": round(w.s, 1), "tol": TOL,
            "value_dtype": w.dtype, "cost": "squared Euclidean / max", "l2": flush,
            "parallelism": "replicas (one independent solve per GPU)"}


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.proc = None
        self.gpu = gpu_index
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={gpu_index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        rows = [r for r in csv.reader(io.StringIO(out)) if len(r) >= 9]
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if r[5 + k].strip().lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _spmv_bytes(res, n, m):
    """Algorithmic HBM bytes of one iteration (row pass + column pass): every
    stored element once (int32 index + value), the pointer arrays, the marginal,
    the old and new scaling vectors, and the gathered vector once."""
    nnz = res["nnz"]
    vb = 4
    row = nnz * (4 + vb) + 4 * (n + 1) + 4 * n * 3 + 4 * m
    col = nnz * (4 + vb) + 4 * (m + 1) + 4 * m * 3 + 4 * n
    return row, col


def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_2306_06581_gb300 import build as _build
    _build.build()
    from paper_2306_06581_gb300 import sparsink as S

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = _workload(args.workload)
    uot = not math.isinf(w.lam)
    dt = torch.float64 if w.dtype == "f64" else torch.float32
    x = torch.tensor(w.x, dtype=dt, device=dev)
    y = torch.tensor(w.y, dtype=dt, device=dev)
    a = torch.tensor(w.a, dtype=dt, device=dev)
    b = torch.tensor(w.b, dtype=dt, device=dev)
    kw = dict(eps=w.eps, s=w.s, tol=TOL, max_iter=20000, dtype=w.dtype, seed=w.seed, problem_id=rank)
    solve = (lambda **extra: S.spar_sink_uot(a, b, x, y, lam=w.lam, **kw, **extra)) if uot else \
        (lambda **extra: S.spar_sink_ot(a, b, x, y, **kw, **extra))
    first = solve()
    ws = first["workspace"]
    flush_buf = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    for _ in range(max(args.warmup, 0)):
        solve(workspace=ws)
    clocks = ClockSampler(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    times, results = [], []
    st = torch.cuda.current_stream()
    for _ in range(args.steps):
        flush_buf.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        r = solve(workspace=ws)
        e1.record(st)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
        results.append(r)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    ms = sum(times) / len(times)
    if world > 1:
        t = torch.tensor([ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    last = results[-1]
    launches = int(sum(r["launches"] for r in results))

    # Roofline of the SpMV half-iterations: a fixed-length run (tol = 0, one
    # chunk, no read-back inside) timed by the library's CUDA events.
    fixed_iters = 200
    kw_fixed = dict(kw, tol=0.0, max_iter=fixed_iters, check_every=fixed_iters)
    if uot:
        rf = S.spar_sink_uot(a, b, x, y, lam=w.lam, **kw_fixed, workspace=ws)
    else:
        rf = S.spar_sink_ot(a, b, x, y, **kw_fixed, workspace=ws)
    row_b, col_b = _spmv_bytes(rf, w.n, w.m)
    per_iter_ms = rf["ms_iter"] / max(rf["iters_enqueued"], 1)
    peak, peak_kind = _peaks()
    achieved = (row_b + col_b) / (per_iter_ms * 1e-3) / 1e9
    traffic = None
    tpath = os.path.join(ROOT, "profiles", f"spmv_traffic_{w.name}.json")
    if os.path.exists(tpath):
        with open(tpath) as f:
            traffic = json.load(f).get("bytes_per_iteration")

    # dense Sinkhorn on the same GPU, same tolerance
    dense = S.sinkhorn_dense(a, b, x, y, eps=w.eps, lam=w.lam, tol=TOL, max_iter=20000, dtype=w.dtype)
    dense = S.sinkhorn_dense(a, b, x, y, eps=w.eps, lam=w.lam, tol=TOL, max_iter=20000, dtype=w.dtype,
                             workspace=dense["workspace"])
    dense_ms = dense["ms_sketch"] + dense["ms_iter"] + dense["ms_obj"]

    # end to end through the public API with host buffers (pinned), copies inside
    hx, hy = torch.tensor(w.x, dtype=dt).pin_memory(), torch.tensor(w.y, dtype=dt).pin_memory()
    ha, hb = torch.tensor(w.a, dtype=dt).pin_memory(), torch.tensor(w.b, dtype=dt).pin_memory()
    e2e = []
    for k in range(max(3, min(args.steps, 20))):
        flush_buf.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        if uot:
            r = S.spar_sink_uot(ha, hb, hx, hy, lam=w.lam, **kw, workspace=ws, device=dev)
        else:
            r = S.spar_sink_ot(ha, hb, hx, hy, **kw, workspace=ws, device=dev)
        al, be = r["alpha"].cpu(), r["beta"].cpu()
        obj = float(r["obj"])
        torch.cuda.synchronize()
        e2e.append((time.perf_counter() - t0) * 1e3)
    h2d = sum(t.numel() * t.element_size() for t in (hx, hy, ha, hb))
    d2h = al.numel() * al.element_size() + be.numel() * be.element_size() + 8 * 16

    line = {
        "metric": METRIC, "value": round(ms, 4), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms, 4), "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32" if w.dtype == "f32" else "f64", "data": "synthetic (seeded)",
        "config": _config(w, "flushed between steps (512 MB write)"),
        "phases_ms": {"sketch": round(last["ms_sketch"], 4), "iterations": round(last["ms_iter"], 4),
                      "objective": round(last["ms_obj"], 4)},
        "iters": last["iters"], "nnz": last["nnz"], "residual": last["residual"], "obj": last["obj"],
        "obj_sparse": last["obj_sparse"],
        "dense_sinkhorn": {"ms": round(dense_ms, 4), "iters": dense["iters"], "obj": dense["obj"],
                           "residual": dense["residual"], "speedup_of_spar_sink": round(dense_ms / ms, 2),
                           "rel_obj_gap_sparse_value": abs(last["obj_sparse"] - dense["obj"]) / abs(dense["obj"])},
        "roofline": {"bound": "hbm", "kernel": "spmv half-iterations (row pass + column pass)",
                     "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(achieved / peak, 4), "peak_kind": peak_kind,
                     "traffic": traffic, "algorithmic_bytes_per_iteration": row_b + col_b,
                     "ms_per_iteration": round(per_iter_ms, 5), "iterations_timed": rf["iters_enqueued"]},
        "e2e": {"value": round(statistics.median(e2e), 4), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": launches,
        "clocks": clk,
    }
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(w)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def _oracle_solve(w):
    import numpy as np

    import oracle
    f = (lambda z: np.asarray(z, np.float32).astype(np.float64)) if w.dtype == "f32" else (lambda z: np.asarray(z))
    P = oracle.OracleProblem(f(w.a), f(w.b), w.eps, w.s, w.lam, x=f(w.x), y=f(w.y), seed=w.seed)
    t0 = time.perf_counter()
    r = oracle.spar_sink(P, tol=TOL, max_iter=20000)
    return (time.perf_counter() - t0) * 1e3, r


def _threads():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_baseline(w):
    import oracle
    oracle.build_oracle()
    ms, r = _oracle_solve(w)
    return {"value": round(ms, 1), "unit": UNIT, "cores": int(os.environ.get("OMP_NUM_THREADS", _threads())),
            "kind": "oracle",
            "sample": f"one complete FP64 oracle solve of {w.name} (sketch, {r['info']['iters']} iterations to "
                      f"1e-5, objective) on the host cores, OpenMP over rows"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    from paper_2306_06581_gb300 import inputs
    oracle.build_oracle()
    w = _workload(args.workload)
    small = inputs.uot_n20000(n=2000) if not math.isinf(w.lam) else inputs.ot_n1000()
    for _ in range(max(args.warmup, 0)):
        _oracle_solve(small)
    times = []
    budget_s = 200.0
    t_start = time.perf_counter()
    for k in range(args.steps):
        ms, r = _oracle_solve(w)
        times.append(ms)
        if (time.perf_counter() - t_start) + ms / 1e3 > budget_s:
            break
    val = sum(times) / len(times)
    cores = int(os.environ.get("OMP_NUM_THREADS", _threads()))
    sample = (f"each step one complete FP64 oracle solve of {w.name} (sketch, iterations to 1e-5, objective); "
              f"{len(times)} of {args.steps} requested steps run within the {budget_s:.0f} s bound; warm-up on n=2000")
    line = {"metric": METRIC, "value": round(val, 1), "unit": UNIT, "n_gpus": int(os.environ.get("WORLD_SIZE", "1")),
            "steps": len(times), "warmup": args.warmup, "ms_per_step": round(val, 1), "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded)",
            "config": _config(w, "n/a (CPU)"), "impl": "reference",
            "cpu_baseline": {"value": round(val, 1), "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": round(val, 1), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="uot_n20000")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
