"""GPU parity at the benchmarked sizes, through the C ABI, against the FP64 oracle.

- The whole 20000-point UOT workload (lambda = 1, R^10, eps = 0.05, skip
  sampler): sketch count equal, objective and sparse-problem value within 1e-5
  relative, iterations within max(3, 3%), potentials element by element after
  the same number of iterations (FP32 bound of parity_util).
- A plain-domain FP32 solve at n = m = 50000 (eps = 0.1): the gathered vector
  (200 KB) no longer fits the plain iteration kernel's shared-memory stage, so
  this runs its unstaged variant; same checks.
- The 1,000,000-point workload (skip sampler, cost divided by its maximum)
  against the stored oracle solve (tests/golden/ot_n1000000_oracle.json,
  written by make_ot_n1000000_oracle.py from the oracle alone): sketch count,
  sampled row and column counts, objective within 1e-5, and the stored
  potentials (gauge sum a alpha = sum b beta) after the oracle's iteration
  count.
- Real pairs of the 64-frame batch (the largest, the smallest and three in
  between), all 2016 pairs solved in one batched call: per pair the sketch
  count, the objective within 1e-5 and the iteration count within max(3, 3%).
"""
import json
import math
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2306_06581_gb300 import inputs  # noqa: E402
from parity_util import compare_potentials, fixed_k, fp32_potential_bound, max_nnz  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def S():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2306_06581_gb300 import build, sparsink
    build.build()
    return sparsink


def _round32(w):
    f = lambda z: np.asarray(z, np.float32).astype(np.float64)
    return f(w.x), f(w.y), f(w.a), f(w.b)


def _iters_close(g, o):
    return abs(g - o) <= max(3, 0.03 * o)


def test_full_uot_n20000_matches_oracle(S, orc):
    w = inputs.uot_n20000()
    x, y, a, b = _round32(w)
    dev = torch.device("cuda")
    xd, yd, ad, bd = (torch.tensor(z, dtype=torch.float32, device=dev) for z in (x, y, a, b))
    run = lambda **e: S.spar_sink_uot(ad, bd, xd, yd, eps=w.eps, lam=w.lam, s=w.s, dtype="f32", seed=w.seed,
                                      sampler="skip", **e)
    g = run(tol=1e-5, max_iter=20000)
    P = orc.OracleProblem(a, b, w.eps, w.s, w.lam, x=x, y=y, seed=w.seed)
    sk = P.sparsify(sampler="skip")
    o = orc.spar_sink(P, tol=1e-5, max_iter=20000, sketch=sk)
    assert g["status"] == 0 and o["info"]["status"] == 0
    assert g["nnz"] == sk["nnz"]
    assert _iters_close(g["iters"], o["info"]["iters"])
    assert abs(g["obj"] - o["obj"]) <= 1e-5 * abs(o["obj"])
    assert abs(g["obj_sparse"] - o["obj_sparse"]) <= 1e-5 * abs(o["obj_sparse"])
    K = o["info"]["iters"]
    gk, ok = fixed_k(run, orc, P, sk, K)
    da, db = compare_potentials(gk["alpha"].cpu(), gk["beta"].cpu(), ok["alpha"], ok["beta"],
                                fp32_potential_bound(w.eps, max_nnz(sk)))
    print(f"UOT n=20000: iters {g['iters']} (oracle {K}), rel obj {abs(g['obj'] - o['obj']) / abs(o['obj']):.1e}, "
          f"max |d alpha| {da:.2e}, |d beta| {db:.2e}")


def test_plain_fp32_n50000_unstaged_matches_oracle(S, orc):
    w = inputs.ot_gmm(50000, d=3, k=8, seed=17, eps=0.1, s_factor=16.0)
    x, y, a, b = _round32(w)
    dev = torch.device("cuda")
    xd, yd, ad, bd = (torch.tensor(z, dtype=torch.float32, device=dev) for z in (x, y, a, b))
    run = lambda **e: S.spar_sink_ot(ad, bd, xd, yd, eps=w.eps, s=w.s, dtype="f32", seed=w.seed, sampler="skip",
                                     **e)
    g = run(tol=1e-5, max_iter=20000)
    P = orc.OracleProblem(a, b, w.eps, w.s, math.inf, x=x, y=y, seed=w.seed)
    sk = P.sparsify(sampler="skip")
    o = orc.spar_sink(P, tol=1e-5, max_iter=20000, sketch=sk)
    assert g["status"] == 0 and o["info"]["status"] == 0
    assert g["nnz"] == sk["nnz"]
    assert _iters_close(g["iters"], o["info"]["iters"])
    assert abs(g["obj"] - o["obj"]) <= 1e-5 * abs(o["obj"])
    K = o["info"]["iters"]
    gk, ok = fixed_k(run, orc, P, sk, K)
    da, db = compare_potentials(gk["alpha"].cpu(), gk["beta"].cpu(), ok["alpha"], ok["beta"],
                                fp32_potential_bound(w.eps, max_nnz(sk)))
    print(f"OT n=50000 plain FP32: iters {g['iters']} (oracle {K}), max |d alpha| {da:.2e}, |d beta| {db:.2e}")


def _gauge_fixed(a, b, al, be):
    fa, fb = np.isfinite(al), np.isfinite(be)
    c = (np.dot(b[fb], be[fb]) - np.dot(a[fa], al[fa])) / 2.0
    return al + c, be - c


def test_n1000000_matches_stored_oracle_solve(S):
    path = os.path.join(HERE, "golden", "ot_n1000000_oracle.json")
    if not os.path.exists(path):
        pytest.skip("stored oracle solve absent (tests/golden/make_ot_n1000000_oracle.py writes it)")
    gold = json.load(open(path))
    w = inputs.ot_n1000000()
    assert gold["workload"] == w.name
    x, y, a, b = _round32(w)
    dev = torch.device("cuda")
    xd, yd, ad, bd = (torch.tensor(z, dtype=torch.float32, device=dev) for z in (x, y, a, b))
    run = lambda **e: S.spar_sink_ot(ad, bd, xd, yd, eps=w.eps, s=w.s, dtype="f32", seed=w.seed, log_domain=1,
                                     sampler="skip", **e)
    g = run(tol=w.tol, max_iter=20000)
    assert g["status"] == 0 and g["nnz"] == gold["nnz"]
    assert _iters_close(g["iters"], gold["iters"])
    assert abs(g["obj"] - gold["obj"]) <= 1e-5 * abs(gold["obj"])
    assert abs(g["obj_sparse"] - gold["obj_sparse"]) <= 1e-5 * abs(gold["obj_sparse"])
    # sampled counts of the sketch
    sk = S.sparsify_kernel(ad, bd, xd, yd, eps=w.eps, s=w.s, dtype="f32", seed=w.seed, sampler="skip")
    rp, cp = sk["row_ptr"].cpu().numpy(), sk["col_ptr"].cpu().numpy()
    for i, c in gold["row_nnz"].items():
        assert rp[int(i) + 1] - rp[int(i)] == c, i
    for j, c in gold["col_nnz"].items():
        assert cp[int(j) + 1] - cp[int(j)] == c, j
    nmax = int(max(np.diff(rp).max(), np.diff(cp).max()))
    del sk
    # potentials after the oracle's iteration count, in the stored gauge
    gk = run(tol=0.0, max_iter=gold["iters"], check_every=gold["iters"], raise_on_error=False)
    assert gk["iters"] == gold["iters"]
    al, be = _gauge_fixed(a, b, gk["alpha"].cpu().numpy().astype(np.float64),
                          gk["beta"].cpu().numpy().astype(np.float64))
    bound = fp32_potential_bound(w.eps, nmax)
    da = max(abs(al[int(i)] - v) for i, v in gold["alpha"].items())
    db = max(abs(be[int(j)] - v) for j, v in gold["beta"].items())
    assert da <= bound and db <= bound, (da, db, bound)
    print(f"OT n=1e6: iters {g['iters']} (oracle {gold['iters']}), rel obj "
          f"{abs(g['obj'] - gold['obj']) / abs(gold['obj']):.1e}, sampled |d alpha| {da:.2e}, |d beta| {db:.2e}")


def test_frames64_pairs_of_one_batch_match_oracle(S, orc):
    sets = inputs.frames()
    pairs = inputs.frame_pairs(len(sets))
    s = [8.0 * inputs.s0(math.sqrt(len(sets[i][1]) * len(sets[j][1]))) for i, j in pairs]
    kw = dict(eps=0.01, lam=1.0, tol=1e-5, max_iter=20000, seed=0x5EED, problem_id=0, cost_norm=S.COST_SCALE,
              cost_scale=inputs.FRAME_COST_SCALE, kdtype="f32")
    r = S.spar_sink_batched(sets, pairs, s, device=torch.device("cuda"), **kw)
    res = r["results"]
    size = np.array([len(sets[i][1]) * len(sets[j][1]) for i, j in pairs], np.float64)
    order = np.argsort(size)
    picks = sorted({int(order[0]), int(order[-1]), int(order[len(order) // 4]), int(order[len(order) // 2]),
                    int(order[3 * len(order) // 4])})
    f = lambda z: np.asarray(z, np.float32).astype(np.float64)
    for p in picks:
        i, j = pairs[p]
        (x, a), (y, b) = sets[i], sets[j]
        P = orc.OracleProblem(f(a), f(b), 0.01, s[p], 1.0, x=f(x), y=f(y), seed=0x5EED, pid=p, cost_norm=2,
                              cost_scale=inputs.FRAME_COST_SCALE)
        o = orc.spar_sink(P, tol=1e-5, max_iter=20000, log_domain=True)
        g = res[p]
        assert g["status"] == 0 and o["info"]["status"] == 0, p
        assert g["nnz"] == o["sketch"]["nnz"], p
        assert _iters_close(g["iters"], o["info"]["iters"]), (p, g["iters"], o["info"]["iters"])
        assert abs(g["obj"] - o["obj"]) <= 1e-5 * abs(o["obj"]), (p, g["obj"], o["obj"])
        print(f"frames pair {p} ({len(a)} x {len(b)}): iters {g['iters']} (oracle {o['info']['iters']}), "
              f"rel obj {abs(g['obj'] - o['obj']) / abs(o['obj']):.1e}")
