"""Benchmark: Spar-Sink time to marginal error 1e-5 vs dense Sinkhorn on one GB300.

A step is one complete Spar-Sink solve of the workload (sketch construction,
scaling iterations until the stopping residual is <= 1e-5, objective), with
the inputs resident in HBM; L2 is flushed (a 512 MB write) between timed steps.
Default workload: balanced OT, n = m = 1,000,000 points in R^3 from
16-component Gaussian mixtures, eps = 0.01 (stabilised iterations with
absorption), s = 16 n ln n, FP32 values and iterates, skip sampler.  The
20000-point UOT workload (lambda = 1, R^10, eps = 0.05) is reported beside it
under "other_workloads"; its sketch stays in L2, so its SpMV rate is labelled
"l2-effective", not HBM.

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


WORKLOADS = ("uot_n20000", "ot_n1000", "ot_n200000", "ot_n1000000", "frames64")


def _frames_batch():
    """64 frames of 96x96, thresholded supports (2.5k-8k pixels), all 2016 pairs
    as UOT (lambda = 1, eps = 0.01), cost = squared pixel distance / (2 95^2),
    s = 8 s0(sqrt(n_i n_j)) per pair."""
    from paper_2306_06581_gb300 import inputs
    sets = inputs.frames()
    pairs = inputs.frame_pairs(len(sets))
    s = [8.0 * inputs.s0(math.sqrt(len(sets[i][1]) * len(sets[j][1]))) for i, j in pairs]
    return sets, pairs, s


def run_batch(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2306_06581_gb300 import build as _build
    from paper_2306_06581_gb300 import inputs
    _build.build()
    from paper_2306_06581_gb300 import sparsink as S

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    sets, pairs, s = _frames_batch()
    kd = args.kdtype or "f32"
    kw = dict(eps=0.01, lam=1.0, tol=TOL, max_iter=20000, seed=0x5EED, problem_id=rank * len(pairs),
              cost_norm=S.COST_SCALE, cost_scale=inputs.FRAME_COST_SCALE, kdtype=kd, sampler=args.sampler)
    dsets = [(torch.tensor(x, dtype=torch.float32, device=dev), torch.tensor(w, dtype=torch.float32, device=dev))
             for x, w in sets]
    stream = torch.cuda.Stream(dev)
    with torch.cuda.stream(stream):
        first = S.spar_sink_batched(dsets, pairs, s, use_graph=1, **kw)
        ws = first["workspace"]
        flush_buf = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
        for _ in range(max(args.warmup, 0)):
            S.spar_sink_batched(dsets, pairs, s, use_graph=1, workspace=ws, **kw)
        clocks = ClockSampler(local)
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        times, last = [], None
        for _ in range(args.steps):
            flush_buf.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            last = S.spar_sink_batched(dsets, pairs, s, use_graph=1, workspace=ws, **kw)
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        clk = clocks.stop()
        # un-captured run for the phase split (sketch vs iterations + objective)
        split = S.spar_sink_batched(dsets, pairs, s, workspace=ws, **kw)
        # the other sampler on the same batch (its own workspace), for the sketch comparison
        other = "element" if args.sampler == "skip" else "skip"
        okw = dict(kw, sampler=other)
        o1 = S.spar_sink_batched(dsets, pairs, s, **okw)
        torch.cuda.synchronize()
        oe0, oe1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        oe0.record(stream)
        o2 = S.spar_sink_batched(dsets, pairs, s, workspace=o1["workspace"], **okw)
        oe1.record(stream)
        oe1.synchronize()
        other_line = {"sampler": other, "ms": round(oe0.elapsed_time(oe1), 3),
                      "phases_ms": {"sketch": round(o2["results"][0]["ms_sketch"], 3),
                                    "iterations_and_objective": round(o2["results"][0]["ms_iter"], 3)},
                      "nnz_total": int(sum(r["nnz"] for r in o2["results"]))}
        del o1, o2
    ms = sum(times) / len(times)
    if world > 1:
        ms = _max_over_ranks(ms, dist, dev)
    res = last["results"]
    iters = np.array([r["iters"] for r in res])
    nnz = np.array([r["nnz"] for r in res], np.float64)
    vb = _VB[kd]
    # algorithmic HBM bytes of the persistent kernel: per pair and iteration one
    # pass over the CSR and one over the CSC (index + value); vectors stay in
    # shared memory; plus the exact first iteration and the objective (log K~
    # and indices, three passes)
    it_bytes = float((iters * nnz * 2 * (4 + vb)).sum() + (nnz * (4 + 4) * 5).sum())
    it_ms = split["results"][0]["ms_iter"]
    peak, peak_kind = _peaks()
    achieved = it_bytes / (it_ms * 1e-3) / 1e9

    # dense Sinkhorn (log-sum-exp form) on the same GPU for a sample of pairs
    samp = list(range(0, len(pairs), max(1, len(pairs) // 8)))[:8]
    dense_ms, dense_it = 0.0, 0
    for p in samp:
        i, j = pairs[p]
        (x, a), (y, b) = dsets[i], dsets[j]
        dkw = dict(eps=0.01, lam=1.0, tol=TOL, max_iter=20000, dtype="f32", cost_norm=S.COST_SCALE,
                   cost_scale=inputs.FRAME_COST_SCALE, log_domain=1, raise_on_error=False)
        dr = S.sinkhorn_dense(a, b, x, y, **dkw)
        dr = S.sinkhorn_dense(a, b, x, y, **dkw, workspace=dr["workspace"])
        dense_ms += dr["ms_sketch"] + dr["ms_iter"] + dr["ms_obj"]
        dense_it += dr["iters"]
    dense_est = dense_ms / len(samp) * len(pairs)

    # end to end through the public API from host arrays
    e2e = []
    for k in range(3):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = S.spar_sink_batched(sets, pairs, s, workspace=ws, device=dev, **kw)
        al, be = r["alpha_flat"].cpu(), r["beta_flat"].cpu()
        torch.cuda.synchronize()
        e2e.append((time.perf_counter() - t0) * 1e3)
    h2d = sum(x.nbytes // 2 + w.nbytes // 2 for x, w in sets)   # float32 copies of the float64 arrays
    d2h = (al.numel() + be.numel()) * 4 + 160 * len(pairs)
    line = {
        "metric": METRIC, "value": round(ms, 3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms, 3), "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": kd, "data": "synthetic (seeded)",
        "config": {"workload": "frames64_pairs2016_uot_lam1_eps0.01", "n_sets": len(sets), "pairs": len(pairs),
                   "support_min": int(min(len(w) for _, w in sets)), "support_max": int(max(len(w) for _, w in sets)),
                   "eps": 0.01, "lambda": 1.0, "tol": TOL, "s": "8 s0(sqrt(n_i n_j)) per pair",
                   "cost": "squared pixel distance / (2 95^2)", "value_dtype": kd, "log_domain": 1,
                   "l2": "flushed between steps (512 MB write)", "graph": "captured once, replayed per step",
                   "parallelism": "replicas (one batch per GPU)", "sampler": args.sampler},
        "pairs_per_s": round(len(pairs) / (ms * 1e-3), 1),
        "other_sampler": other_line,
        "phases_ms": {"sketch": round(split["results"][0]["ms_sketch"], 3), "iterations_and_objective": round(it_ms, 3)},
        "iters": {"mean": float(iters.mean()), "max": int(iters.max()), "min": int(iters.min())},
        "not_converged": int(sum(r["status"] != 0 for r in res)), "nnz_total": int(nnz.sum()),
        "launch_shape": {"lanes_per_row": first["lanes_per_row"], "block_threads": first["block_threads"],
                         "tune_ms": round(first["tune_ms"], 1)},
        "dense_sinkhorn": {"sample_pairs": len(samp), "sample_ms": round(dense_ms, 2),
                           "mean_iters": dense_it / len(samp), "log_domain": 1,
                           "extrapolated_ms_all_pairs": round(dense_est, 1),
                           "speedup_of_spar_sink_extrapolated": round(dense_est / ms, 2)},
        "roofline": {"bound": "hbm", "kernel": "persistent batched iterations (CSR + CSC passes per iteration)",
                     "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s", "frac": round(achieved / peak, 4),
                     "peak_kind": peak_kind, "traffic": None, "algorithmic_bytes": it_bytes},
        "e2e": {"value": round(statistics.median(e2e), 3), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": 14 * args.steps,
        "clocks": clk,
    }
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = _batch_cpu_baseline(sets, pairs, s, sampler=args.sampler)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def _batch_cpu_baseline(sets, pairs, s, k=2, sampler="element"):
    import numpy as np

    import oracle
    from paper_2306_06581_gb300 import inputs
    oracle.build_oracle()
    samp = list(range(0, len(pairs), max(1, len(pairs) // k)))[:k]
    t0 = time.perf_counter()
    for p in samp:
        i, j = pairs[p]
        (x, a), (y, b) = sets[i], sets[j]
        f = lambda z: np.asarray(z, np.float32).astype(np.float64)
        P = oracle.OracleProblem(f(a), f(b), 0.01, s[p], 1.0, x=f(x), y=f(y), seed=0x5EED, pid=p,
                                 cost_norm=2, cost_scale=inputs.FRAME_COST_SCALE)
        oracle.spar_sink(P, tol=TOL, max_iter=20000, log_domain=True, sketch=P.sparsify(sampler=sampler))
    el = (time.perf_counter() - t0) * 1e3
    return {"value": round(el / len(samp) * len(pairs), 1), "unit": UNIT,
            "cores": int(os.environ.get("OMP_NUM_THREADS", _threads())), "kind": "oracle",
            "sample": f"FP64 oracle Spar-Sink (log domain, {sampler} sampler) of {len(samp)} of the {len(pairs)} "
                      f"pairs, {el / 1e3:.1f} s, scaled to all pairs"}


def _workload(name, n=None):
    """The named workload; n (profiling) re-draws the same family at another size."""
    from paper_2306_06581_gb300 import inputs
    kw = {} if n is None else {"n": n}
    if name == "uot_n20000":
        return inputs.uot_n20000(**kw)
    if name == "ot_n1000":
        return inputs.ot_n1000(**kw)
    if name == "ot_n200000":
        return inputs.ot_n200000(**kw)
    if name == "ot_n1000000":
        return inputs.ot_n1000000(**kw)
    raise SystemExit(f"unknown workload {name}")


def _log_domain(w):
    """The stabilised iterations run for eps < 0.05 (K~ leaves the binary32 range)."""
    return 1 if w.eps < 0.05 else 0


def _problem_dtype(w):
    return "f64" if w.dtype == "f64" else "f32"


def _config(w, flush, kdtype=None):
    return {"workload": w.name, "n": w.n, "m": w.m, "d": w.d, "eps": w.eps,
            "lambda": None if math.isinf(w.lam) else w.lam, "s": round(w.s, 1), "tol": TOL,
            "value_dtype": kdtype or w.dtype, "log_domain": _log_domain(w), "cost": "squared Euclidean / max",
            "l2": flush, "parallelism": "replicas (one independent solve per GPU)"}


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


_VB = {"f64": 8, "f32": 4, "bf16": 2, "f16": 2}


def _max_over_ranks(x, dist, device):
    """The slowest rank's value (replicas: every rank times its own solve)."""
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _kernel_ms_per_iteration(res, log_domain):
    """Device time of one iteration of the iteration kernel: the solve's
    iteration phase less its setup (the initial pair; in the log domain the
    exact first iteration, the absorption and the grouped copies), over the
    iterations the kernel ran (the first log-domain iteration is the setup's)."""
    its = res["iters_enqueued"] - (1 if log_domain else 0)
    return (res["ms_iter"] - res["ms_setup"]) / max(its, 1)


def _spmv_bytes(res, n, m, kdtype="f32", log_domain=0):
    """Algorithmic HBM bytes of one iteration (row pass + column pass): every
    stored element once (int32 index + value), the pointer arrays, the per-row
    vectors (plain: marginal, old and new scaling; stabilised: also the
    absorbed marginal and the row exponent), and the gathered vector once."""
    nnz = res["nnz"]
    vb = _VB[kdtype]
    ib = 8 if kdtype == "f64" else 4
    kr = 5 if log_domain else 3
    kc = 4 if log_domain else 3
    row = nnz * (4 + vb) + 4 * (n + 1) + ib * n * kr + ib * m
    col = nnz * (4 + vb) + 4 * (m + 1) + ib * m * kc + ib * n
    return row, col


def _stream_bytes(res, n, m, kdtype="f32", log_domain=0):
    """Bytes one iteration streams when the staged passes read the grouped
    copies (sps_result.stream_bytes: both copies, with their headers and
    padding, 16-bit indices) plus the same per-row and per-column vectors as
    _spmv_bytes; None when the solve gathered directly."""
    if not res.get("stream_bytes"):
        return None
    row, col = _spmv_bytes(res, n, m, kdtype, log_domain)
    vectors = row + col - 2 * res["nnz"] * (4 + _VB[kdtype]) - 4 * (n + 1) - 4 * (m + 1)
    return int(res["stream_bytes"] + vectors)


def _stream_fields(res, w, kd, logd, per_iter_ms, peak):
    """The staged passes' own bytes next to the algorithmic ones: what one
    iteration streams (grouped copies, 16-bit indices) and the fraction of the
    peak that rate is; empty when the solve gathered directly."""
    sb = _stream_bytes(res, w.n, w.m, kd, logd)
    if sb is None:
        return {}
    rate = sb / (per_iter_ms * 1e-3) / 1e9
    return {"stream_bytes_per_iteration": sb, "stream_gbs": round(rate, 1), "stream_frac": round(rate / peak, 4)}


def _traffic(name):
    """DRAM bytes per iteration of the iteration kernel from the committed ncu
    summary of this workload (profiles/spmv_traffic_<name>.txt): (bytes, the
    summary's file name), or (None, None)."""
    fn = f"spmv_traffic_{name}.txt"
    p = os.path.join(ROOT, "profiles", fn)
    if not os.path.exists(p):
        return None, None
    with open(p) as f:
        for line in f:
            if line.startswith("bytes_per_iteration:"):
                return float(line.split(":", 1)[1]), "profiles/" + fn
    return None, None


def _bound(traffic, algorithmic):
    """HBM-bound only when the DRAM traffic measured for the kernel is at least
    half of its algorithmic bytes; a sketch that stays in L2 reads far less
    from DRAM, and its rate is an L2-effective one."""
    if traffic is None:
        return "hbm (traffic not measured)"
    return "hbm" if traffic >= 0.5 * algorithmic else "l2-effective"


def _dense_cap(args, w):
    """Dense Sinkhorn iterations allowed before the run stops and its time to
    tolerance is extrapolated: --dense-cap if given (> 0), else 2 above 1e10
    kernel entries (a dense iteration at n = m = 10^6 takes about 2 s), else no cap."""
    if args.dense_cap > 0:
        return args.dense_cap
    return 2 if float(w.n) * w.m > 1e10 else 20000


def _golden(w):
    """FP64 oracle result of the workload stored by tests/golden (None if absent)."""
    p = os.path.join(ROOT, "tests", "golden", f"{w.name.split('_d')[0]}_oracle.json")
    if os.path.exists(p):
        with open(p) as f:
            g = json.load(f)
        if g.get("workload") == w.name:
            return g
    return None


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
    w = _workload(args.workload, args.n)
    uot = not math.isinf(w.lam)
    pdt = _problem_dtype(w)
    kd = args.kdtype or w.dtype
    logd = _log_domain(w)
    dt = torch.float64 if pdt == "f64" else torch.float32
    x = torch.tensor(w.x, dtype=dt, device=dev)
    y = torch.tensor(w.y, dtype=dt, device=dev)
    a = torch.tensor(w.a, dtype=dt, device=dev)
    b = torch.tensor(w.b, dtype=dt, device=dev)
    kw = dict(eps=w.eps, s=w.s, tol=TOL, max_iter=20000, dtype=pdt, seed=w.seed, problem_id=rank)

    def solve(**extra):
        k = dict(kw, kdtype=kd, log_domain=logd, sampler=args.sampler)
        k.update(extra)
        if uot:
            return S.spar_sink_uot(k.pop("a", a), k.pop("b", b), k.pop("x", x), k.pop("y", y), lam=w.lam, **k)
        return S.spar_sink_ot(k.pop("a", a), k.pop("b", b), k.pop("x", x), k.pop("y", y), **k)

    first = solve()
    ws = first["workspace"]
    if args.solve_only:
        # one more solve in the same workspace, for profilers; no timing loop
        r = solve(workspace=ws)
        if rank == 0:
            print(json.dumps({"workload": w.name, "iters": r["iters"], "nnz": r["nnz"], "obj": r["obj"],
                              "ms": r["ms_sketch"] + r["ms_iter"] + r["ms_obj"]}), flush=True)
        return
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
        ms = _max_over_ranks(ms, dist, dev)
    last = results[-1]
    launches = int(sum(r["launches"] for r in results))

    # Roofline of the SpMV half-iterations: a fixed-length run (tol = 0, one
    # chunk, no read-back inside) timed by the library's CUDA events.
    fixed_iters = 200
    rf = solve(tol=0.0, max_iter=fixed_iters, check_every=fixed_iters, workspace=ws)
    row_b, col_b = _spmv_bytes(rf, w.n, w.m, kd, logd)
    per_iter_ms = _kernel_ms_per_iteration(rf, logd)
    peak, peak_kind = _peaks()
    achieved = (row_b + col_b) / (per_iter_ms * 1e-3) / 1e9
    traffic, traffic_src = _traffic(w.name)

    # dense Sinkhorn on the same GPU, same tolerance (log-sum-exp form for small
    # eps); with --dense-cap the run stops after that many iterations and the
    # time to tolerance is extrapolated at Spar-Sink's iteration count
    cap = _dense_cap(args, w)
    dkw = dict(eps=w.eps, lam=w.lam, tol=TOL, max_iter=cap, dtype=pdt, log_domain=logd, raise_on_error=False)
    dense = S.sinkhorn_dense(a, b, x, y, **dkw)
    dense = S.sinkhorn_dense(a, b, x, y, **dkw, workspace=dense["workspace"])
    dense_ms = dense["ms_sketch"] + dense["ms_iter"] + dense["ms_obj"]
    dense_line = {"ms": round(dense_ms, 4), "iters": dense["iters"], "obj": dense["obj"],
                  "residual": dense["residual"], "log_domain": logd}
    if dense["status"] == 0:
        dense_line["speedup_of_spar_sink"] = round(dense_ms / ms, 2)
        dense_line["rel_obj_gap_sparse_value"] = abs(last["obj_sparse"] - dense["obj"]) / abs(dense["obj"])
    else:
        per = dense["ms_iter"] / max(dense["iters_enqueued"], 1)
        est = dense["ms_sketch"] + per * last["iters"] + dense["ms_obj"]
        dense_line.update({"capped_at_iters": cap, "ms_per_iteration": round(per, 4),
                           "extrapolated_ms_at_spar_sink_iters": round(est, 1),
                           "speedup_of_spar_sink_extrapolated": round(est / ms, 2)})

    # the same solve with the other sampler (same law, another random stream)
    other = None
    if rank == 0:
        alt = "skip" if args.sampler == "element" else "element"
        ro = solve(sampler=alt)
        tms = []
        for _ in range(3):
            flush_buf.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            ro = solve(sampler=alt, workspace=ro["workspace"])
            e1.record(st)
            e1.synchronize()
            tms.append(e0.elapsed_time(e1))
        other = {"sampler": alt, "ms": round(sum(tms) / len(tms), 4),
                 "phases_ms": {"sketch": round(ro["ms_sketch"], 4), "iterations": round(ro["ms_iter"], 4),
                               "objective": round(ro["ms_obj"], 4)},
                 "iters": ro["iters"], "nnz": ro["nnz"], "obj": ro["obj"],
                 "rel_obj_diff": abs(ro["obj"] - last["obj"]) / abs(last["obj"])}

    # storage precision forms of the stabilised path against the stored FP64 oracle value
    precision = None
    gold = _golden(w)
    if logd and rank == 0 and gold is not None:
        precision = {}
        gs = gold.get("sampler", "element")   # the stream the stored oracle solve was sketched with
        for k2 in ("f32", "bf16", "f16"):
            rr = solve(kdtype=k2, sampler=gs)
            rr = solve(kdtype=k2, sampler=gs, workspace=rr["workspace"])
            ent = {"ms": round(rr["ms_sketch"] + rr["ms_iter"] + rr["ms_obj"], 3), "iters": rr["iters"],
                   "obj": rr["obj"], "n_absorb": rr["n_absorb"]}
            if gold is not None:
                ent["rel_err_vs_fp64_oracle"] = abs(rr["obj"] - gold["obj"]) / abs(gold["obj"])
                ent["oracle_iters"] = gold["iters"]
                ent["sampler"] = gs
            precision[k2] = ent

    # end to end through the public API with host buffers (pinned), copies inside
    hx, hy = torch.tensor(w.x, dtype=dt).pin_memory(), torch.tensor(w.y, dtype=dt).pin_memory()
    ha, hb = torch.tensor(w.a, dtype=dt).pin_memory(), torch.tensor(w.b, dtype=dt).pin_memory()
    e2e = []
    for k in range(max(3, min(args.steps, 20))):
        flush_buf.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = solve(a=ha, b=hb, x=hx, y=hy, workspace=ws, device=dev)
        al, be = r["alpha"].cpu(), r["beta"].cpu()
        obj = float(r["obj"])
        torch.cuda.synchronize()
        e2e.append((time.perf_counter() - t0) * 1e3)
    h2d = sum(t.numel() * t.element_size() for t in (hx, hy, ha, hb))
    d2h = al.numel() * al.element_size() + be.numel() * be.element_size() + 8 * 16

    line = {
        "metric": METRIC, "value": round(ms, 4), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms, 4), "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": kd, "data": "synthetic (seeded)",
        "config": _config(w, "flushed between steps (512 MB write)", kd),
        "phases_ms": {"sketch": round(last["ms_sketch"], 4), "iterations": round(last["ms_iter"], 4),
                      "objective": round(last["ms_obj"], 4)},
        "iters": last["iters"], "nnz": last["nnz"], "residual": last["residual"], "obj": last["obj"],
        "obj_sparse": last["obj_sparse"], "n_absorb": last["n_absorb"],
        "dense_sinkhorn": dense_line,
        "roofline": {"bound": _bound(traffic, row_b + col_b),
                     "kernel": "spmv half-iterations (row pass + column pass)",
                     "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(achieved / peak, 4), "peak_kind": peak_kind,
                     "traffic": traffic, "traffic_source": traffic_src,
                     "algorithmic_bytes_per_iteration": row_b + col_b,
                     "ms_per_iteration": round(per_iter_ms, 5), "iterations_timed": rf["iters_enqueued"],
                     **_stream_fields(rf, w, kd, logd, per_iter_ms, peak)},
        "e2e": {"value": round(statistics.median(e2e), 4), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": launches,
        "clocks": clk,
    }
    line["config"]["sampler"] = args.sampler
    if other is not None:
        line["other_sampler"] = other
    if precision is not None:
        line["precision_forms"] = precision
    if rank == 0 and not args.no_other_workloads:
        others = {}
        for name in ("uot_n20000",):
            if name != w.name.split("_d")[0]:
                others[name] = _other_workload_leg(S, name, dev, flush_buf, args.sampler)
        line["other_workloads"] = others
    if args.warm_start:
        line["warm_start"] = _warm_start_leg(args, w, S, x, y, a, b, kd, logd, last)
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(w, args.sampler)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def _other_workload_leg(S, name, dev, flush_buf, sampler, steps=10):
    """Time per solve of another named workload (inputs resident, L2 flushed
    between solves), with the SpMV rate of a fixed 200-iteration run labelled
    by the DRAM traffic measured for it."""
    import torch
    w = _workload(name)
    pdt = _problem_dtype(w)
    dt = torch.float64 if pdt == "f64" else torch.float32
    x, y, a, b = (torch.tensor(z, dtype=dt, device=dev) for z in (w.x, w.y, w.a, w.b))
    kd, logd = w.dtype, _log_domain(w)
    kw = dict(eps=w.eps, s=w.s, tol=TOL, max_iter=20000, dtype=pdt, kdtype=kd, seed=w.seed, log_domain=logd,
              sampler=sampler)
    if math.isinf(w.lam):
        run = lambda **e: S.spar_sink_ot(a, b, x, y, **dict(kw, **e))
    else:
        run = lambda **e: S.spar_sink_uot(a, b, x, y, lam=w.lam, **dict(kw, **e))
    r = run()
    ws = r["workspace"]
    for _ in range(3):
        run(workspace=ws)
    st = torch.cuda.current_stream()
    times = []
    for _ in range(steps):
        flush_buf.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        r = run(workspace=ws)
        e1.record(st)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    rf = run(tol=0.0, max_iter=200, check_every=200, workspace=ws)
    row_b, col_b = _spmv_bytes(rf, w.n, w.m, kd, logd)
    per = _kernel_ms_per_iteration(rf, logd)
    peak, peak_kind = _peaks()
    ach = (row_b + col_b) / (per * 1e-3) / 1e9
    traffic, src = _traffic(w.name)
    return {"workload": w.name, "ms": round(sum(times) / len(times), 4), "steps": steps,
            "phases_ms": {"sketch": round(r["ms_sketch"], 4), "iterations": round(r["ms_iter"], 4),
                          "objective": round(r["ms_obj"], 4)},
            "iters": r["iters"], "nnz": r["nnz"], "obj": r["obj"],
            "roofline": {"bound": _bound(traffic, row_b + col_b), "achieved": round(ach, 1), "peak": peak,
                         "unit": "GB/s", "frac": round(ach / peak, 4), "peak_kind": peak_kind,
                         "traffic": traffic, "traffic_source": src,
                         "algorithmic_bytes_per_iteration": row_b + col_b, "ms_per_iteration": round(per, 5),
                         **_stream_fields(rf, w, kd, logd, per, peak)}}


def _warm_start_leg(args, w, S, x, y, a, b, kd, logd, cold):
    """Train the warm-start network on seeded smaller instances of the same
    family (targets from the solver), then time warm-started Spar-Sink on the
    workload: exact cost divisor + inference + solve, against the cold solve."""
    import torch

    from paper_2306_06581_gb300 import inputs
    from paper_2306_06581_gb300 import warmstart as WS
    t0 = time.perf_counter()
    data = []
    for k in range(args.ws_instances):
        wk = inputs.ot_gmm16(args.ws_n, seed=1000 + k)
        inst, al, be, _ = WS.solve_targets(wk, w.eps, wk.s, seed=wk.seed, kdtype=kd, sampler=args.sampler)
        data.append((inst, al, be))
    t1 = time.perf_counter()
    net = WS.WarmStart(w.d, seed=5)
    losses = WS.train(net, data, args.ws_steps, lr=2e-3, lr_end=2e-4)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    st = torch.cuda.current_stream()
    kw = dict(eps=w.eps, s=w.s, tol=TOL, max_iter=20000, dtype="f32", kdtype=kd, seed=w.seed, log_domain=logd,
              sampler=args.sampler)
    runs = []
    for rep in range(2):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        cm = S.cost_max(x, y)
        al, be = net.predict(net.instance(x, a, y, b, cm))
        r = S.spar_sink_ot(a, b, x, y, init_alpha=al, init_beta=be, cost_norm=S.COST_SCALE, cost_scale=cm, **kw)
        e1.record(st)
        e1.synchronize()
        runs.append((e0.elapsed_time(e1), r))
    ms, r = runs[-1]
    # the exact cost divisor alone (it synchronises), then the network's inference alone (both sides)
    tc = time.perf_counter()
    cm = S.cost_max(x, y)
    cm_ms = (time.perf_counter() - tc) * 1e3
    inst = net.instance(x, a, y, b, cm)
    net.predict(inst)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(5):
        net.predict(inst)
    e1.record(st)
    e1.synchronize()
    inf_ms = e0.elapsed_time(e1) / 5
    return {"ms": round(ms, 3), "sampler": args.sampler, "iters": r["iters"], "cold_iters": cold["iters"],
            "cost_max_ms": round(cm_ms, 3), "inference_ms": round(inf_ms, 3),
            "inference_share": round(inf_ms / ms, 4),
            "obj_rel_diff_vs_cold": abs(r["obj"] - cold["obj"]) / abs(cold["obj"]),
            "ms_iterations": round(r["ms_iter"], 3), "cold_ms_iterations": round(cold["ms_iter"], 3),
            "training": {"instances": args.ws_instances, "n": args.ws_n, "steps": args.ws_steps,
                         "targets_s": round(t1 - t0, 1), "train_s": round(t2 - t1, 1),
                         "loss_first": float(sum(losses[:64]) / len(losses[:64])),
                         "loss_last": float(sum(losses[-64:]) / len(losses[-64:]))},
            "includes": "exact cost divisor, network inference and the solve (cold: the solve, which finds the divisor itself)"}


def _f32(z):
    import numpy as np
    return np.asarray(z, np.float32).astype(np.float64)


def _oracle_problem(w, rows=None):
    import oracle
    f = _f32 if w.dtype != "f64" else (lambda z: z)
    x = w.x if rows is None else w.x[:rows]
    a = w.a if rows is None else w.a[:rows]
    # a row subset keeps the per-element probabilities of the whole problem with s scaled by rows/n
    s = w.s if rows is None else w.s * rows / w.n
    return oracle.OracleProblem(f(a), f(w.b), w.eps, s, w.lam, x=f(x), y=f(w.y), seed=w.seed)


def _oracle_solve(w, sampler="element"):
    import oracle
    P = _oracle_problem(w)
    t0 = time.perf_counter()
    r = oracle.spar_sink(P, tol=TOL, max_iter=20000, log_domain=bool(_log_domain(w)),
                         sketch=P.sparsify(sampler=sampler))
    return (time.perf_counter() - t0) * 1e3, r


# a full oracle solve above this many decisions (n m) is replaced by a bounded sample
FULL_ORACLE_MAX_PAIRS = 1.0e9


def _oracle_sampled(w, rows, iters, gold_iters, sampler="element"):
    """Bounded oracle sample of a large workload: the sketch (cost maximum,
    count and fill passes) of the first `rows` rows against all m columns,
    `iters` iterations and the objective on that partial sketch.  Returns the
    whole-solve estimate (sketch scaled by n/rows, iterations and objective by
    the nnz ratio and the iteration count) in ms, and a description."""
    import oracle
    P = _oracle_problem(w, rows)
    t0 = time.perf_counter()
    sk = P.sparsify(sampler=sampler)
    t1 = time.perf_counter()
    it = oracle.spar_sink(P, tol=0.0, max_iter=iters, log_domain=bool(_log_domain(w)), sketch=sk)
    t2 = time.perf_counter()
    nnz_full = w.s  # expected nnz of the whole sketch (no clipping at these budgets)
    scale = nnz_full / max(sk["nnz"], 1)
    per_iter = (t2 - t1) / max(iters, 1)   # includes the objective pass once per `iters` iterations
    est = ((t1 - t0) * w.n / rows + per_iter * scale * gold_iters) * 1e3
    desc = (f"FP64 oracle on the first {rows} of {w.n} rows against all {w.m} columns: sketch "
            f"{(t1 - t0):.1f} s scaled by n/rows, then {iters} iterations + objective on that partial sketch "
            f"({sk['nnz']} of ~{int(nnz_full)} elements) scaled by the element count to {gold_iters} iterations")
    return est, desc


def _threads():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


_THREADING = ("the oracle's cost maximum, UOT normaliser and sketch run on all host cores (OpenMP over rows); "
              "its iterations and objective run on one thread")
_THREADING_1 = "every part of the oracle runs on one thread (OpenMP limited to 1)"


def _omp_set_threads(k):
    """Thread count of the OpenMP runtime the oracle is linked with (False if
    the runtime cannot be reached)."""
    import ctypes
    try:
        ctypes.CDLL("libgomp.so.1").omp_set_num_threads(int(k))
        return True
    except (OSError, AttributeError):
        return False


def _baseline_sample(w, sampler="element", scale=1):
    """The oracle timed on a bounded sample of the workload; scale > 1 shrinks
    the sample (fewer rows) for the one-thread configuration."""
    threading = _THREADING if scale == 1 else _THREADING_1
    if float(w.n) * w.m <= FULL_ORACLE_MAX_PAIRS and scale == 1:
        ms, r = _oracle_solve(w, sampler)
        return ms, (f"one complete FP64 oracle solve of {w.name} ({sampler} sampler sketch, {r['info']['iters']} "
                    f"iterations to 1e-5, objective); {threading}")
    gold = _golden(w)
    gi = gold["iters"] if gold else 200
    rows = max(256 // scale, int(4.0e8 / w.m) // scale, 16)
    if float(w.n) * w.m <= FULL_ORACLE_MAX_PAIRS:
        rows = max(16, w.n // (8 * scale))
    est, desc = _oracle_sampled(w, rows, 5, gi, sampler)
    return est, desc + "; " + threading


def cpu_baseline(w, sampler="element"):
    import oracle
    oracle.build_oracle()
    ms, desc = _baseline_sample(w, sampler)
    out = {"value": round(ms, 1), "unit": UNIT, "cores": int(os.environ.get("OMP_NUM_THREADS", _threads())),
           "kind": "oracle", "sample": desc}
    # the same oracle on one thread, on a sample 8 times smaller, scaled the same way
    if _omp_set_threads(1):
        try:
            ms1, desc1 = _baseline_sample(w, sampler, scale=8)
            out["one_thread"] = {"value": round(ms1, 1), "unit": UNIT, "cores": 1, "sample": desc1}
        finally:
            _omp_set_threads(out["cores"])
    return out


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    from paper_2306_06581_gb300 import inputs
    oracle.build_oracle()
    if args.workload == "frames64":
        sets, pairs, s = _frames_batch()
        times = []
        t_start = time.perf_counter()
        for k in range(args.steps):
            b = _batch_cpu_baseline(sets, pairs, s, sampler=args.sampler)
            times.append(b["value"])
            if time.perf_counter() - t_start > 200.0:
                break
        val = sum(times) / len(times)
        line = {"metric": METRIC, "value": round(val, 1), "unit": UNIT,
                "n_gpus": int(os.environ.get("WORLD_SIZE", "1")), "steps": len(times), "warmup": args.warmup,
                "ms_per_step": round(val, 1), "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
                "dtype": "f64", "data": "synthetic (seeded)",
                "config": {"workload": "frames64_pairs2016_uot_lam1_eps0.01"}, "impl": "reference",
                "cpu_baseline": dict(b, value=round(val, 1)),
                "e2e": {"value": round(val, 1), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return
    w = _workload(args.workload)
    small = inputs.uot_n20000(n=2000) if not math.isinf(w.lam) else inputs.ot_n1000()
    for _ in range(max(args.warmup, 0)):
        _oracle_solve(small)
    times, descs = [], []
    budget_s = 200.0
    t_start = time.perf_counter()
    for k in range(args.steps):
        t0 = time.perf_counter()
        ms, desc = _baseline_sample(w, args.sampler)
        times.append(ms)
        descs.append(desc)
        if (time.perf_counter() - t_start) + (time.perf_counter() - t0) > budget_s:
            break
    val = sum(times) / len(times)
    cores = int(os.environ.get("OMP_NUM_THREADS", _threads()))
    sample = (f"each step: {descs[-1]}; {len(times)} of {args.steps} requested steps run within the "
              f"{budget_s:.0f} s bound; warm-up on a small instance")
    line = {"metric": METRIC, "value": round(val, 1), "unit": UNIT, "n_gpus": int(os.environ.get("WORLD_SIZE", "1")),
            "steps": len(times), "warmup": args.warmup, "ms_per_step": round(val, 1), "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded)",
            "config": _config(w, "n/a (CPU)", args.kdtype or w.dtype), "impl": "reference",
            "cpu_baseline": {"value": round(val, 1), "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": round(val, 1), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    line["config"]["sampler"] = args.sampler
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="ot_n1000000", choices=WORKLOADS)
    ap.add_argument("--kdtype", default=None, choices=["f64", "f32", "bf16", "f16"],
                    help="storage type of the sketch values (default: the workload's)")
    ap.add_argument("--dense-cap", type=int, default=0,
                    help="stop dense Sinkhorn after this many iterations and extrapolate "
                         "(0: 2 above 1e10 kernel entries, else run to tolerance)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-other-workloads", action="store_true", help="skip the 20000-point UOT leg")
    ap.add_argument("--sampler", default="skip", choices=["element", "skip"],
                    help="sketch draws: geometric skips with thinning (default), or one decision per element")
    ap.add_argument("--n", type=int, default=None, help="profiling: the workload's family at another size")
    ap.add_argument("--solve-only", action="store_true", help="profiling: two solves, no timing loop")
    ap.add_argument("--warm-start", action="store_true", help="also train and time the learned warm start")
    ap.add_argument("--ws-instances", type=int, default=512)
    ap.add_argument("--ws-n", type=int, default=50000)
    ap.add_argument("--ws-steps", type=int, default=2000)
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "frames64":
        run_batch(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
