"""GPU checks of the batched solver (many pairs over shared point sets, one
persistent launch): each pair equals a single-problem solve with the same
Philox problem id, and the FP64 oracle's Alg. 4 / Alg. 3 in log form."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2306_06581_gb300 import build, sparsink
    build.build()
    return sparsink


def _sets(seed, sizes, d=2, span=40.0):
    rng = np.random.default_rng(seed)
    out = []
    for k, n in enumerate(sizes):
        c = rng.uniform(0, span, d)
        x = (c + rng.normal(0, span / 6, (n, d))).astype(np.float32).astype(np.float64)
        w = rng.uniform(0.2, 1.0, n)
        w = (w / w.sum() * rng.uniform(0.8, 1.2)).astype(np.float32).astype(np.float64)
        out.append((x, w))
    return out


SCALE = 2.0 * 60.0 ** 2


def _pairs(k):
    return [(i, j) for i in range(k) for j in range(i + 1, k)]


@pytest.fixture(scope="module")
def uot_batch(S):
    sets = _sets(5, [420, 650, 300, 520, 800])
    pairs = _pairs(5)
    s = [12.0 * math.sqrt(len(sets[i][1]) * len(sets[j][1])) * math.log(len(sets[i][1])) for i, j in pairs]
    kw = dict(eps=0.01, lam=1.0, tol=1e-5, max_iter=5000, seed=77, problem_id=3,
              cost_norm=S.COST_SCALE, cost_scale=SCALE)
    r = S.spar_sink_batched(sets, pairs, s, **kw)
    return sets, pairs, s, kw, r


def test_batch_pairs_equal_single_solves(S, uot_batch):
    sets, pairs, s, kw, r = uot_batch
    assert r["status_code"] == 0
    for p, (i, j) in enumerate(pairs):
        (x, a), (y, b) = sets[i], sets[j]
        g = S.spar_sink_uot(a, b, x, y, eps=kw["eps"], lam=1.0, s=s[p], tol=kw["tol"], max_iter=5000, dtype="f32",
                            seed=kw["seed"], problem_id=kw["problem_id"] + p, cost_norm=S.COST_SCALE,
                            cost_scale=SCALE, log_domain=1)
        rb = r["results"][p]
        assert rb["status"] == 0 and rb["nnz"] == g["nnz"], p
        assert abs(rb["iters"] - g["iters"]) <= max(2, 0.03 * g["iters"]), (p, rb["iters"], g["iters"])
        assert abs(rb["obj"] - g["obj"]) <= 2e-6 * abs(g["obj"]), p
        assert torch.allclose(r["alpha"][p], g["alpha"], rtol=0, atol=2e-5)


def test_batch_pairs_match_oracle(S, orc, uot_batch):
    sets, pairs, s, kw, r = uot_batch
    for p in (0, 4, 9):
        i, j = pairs[p]
        (x, a), (y, b) = sets[i], sets[j]
        P = orc.OracleProblem(a, b, kw["eps"], s[p], 1.0, x=x, y=y, seed=kw["seed"], pid=kw["problem_id"] + p,
                              cost_norm=S.COST_SCALE, cost_scale=SCALE)
        o = orc.spar_sink(P, tol=kw["tol"], max_iter=5000, log_domain=True)
        rb = r["results"][p]
        assert rb["nnz"] == o["sketch"]["nnz"], p
        assert abs(rb["iters"] - o["info"]["iters"]) <= max(3, 0.05 * o["info"]["iters"]), p
        assert abs(rb["obj"] - o["obj"]) <= 1e-5 * abs(o["obj"]), p
        for k in ("kl_a", "kl_b", "mass"):
            assert abs(rb[k] - o["terms"][k]) <= 1e-4 * abs(o["terms"][k]) + 1e-9, (p, k)


def test_batch_ot_matches_oracle(S, orc):
    # balanced OT: every set carries unit mass
    sets = [(x, (w / w.sum()).astype(np.float32).astype(np.float64)) for x, w in _sets(6, [350, 500, 610])]
    pairs = [(0, 1), (1, 2), (2, 0), (1, 1)]
    s = [8000.0, 12000.0, 9000.0, 15000.0]
    r = S.spar_sink_batched(sets, pairs, s, eps=0.02, tol=1e-5, max_iter=5000, seed=5, cost_norm=S.COST_MAXNORM)
    assert r["status_code"] == 0
    for p, (i, j) in enumerate(pairs):
        (x, a), (y, b) = sets[i], sets[j]
        P = orc.OracleProblem(a, b, 0.02, s[p], math.inf, x=x, y=y, seed=5, pid=p)
        o = orc.spar_sink(P, tol=1e-5, max_iter=5000, log_domain=True)
        rb = r["results"][p]
        assert rb["nnz"] == o["sketch"]["nnz"], p
        assert abs(rb["obj"] - o["obj"]) <= 1e-5 * abs(o["obj"]) + 1e-7, (p, rb["obj"], o["obj"])


def test_batch_graph_replay_and_shapes(S, uot_batch):
    sets, pairs, s, kw, r = uot_batch
    g1 = S.spar_sink_batched(sets, pairs, s, use_graph=1, **kw)
    g2 = S.spar_sink_batched(sets, pairs, s, use_graph=1, workspace=g1["workspace"], **kw)
    g3 = S.spar_sink_batched(sets, pairs, s, use_graph=1, workspace=g1["workspace"], **kw)
    for a_, b_ in ((g2, g3),):
        assert [x["iters"] for x in a_["results"]] == [x["iters"] for x in b_["results"]]
        assert [x["obj"] for x in a_["results"]] == [x["obj"] for x in b_["results"]]
        assert torch.equal(a_["alpha_flat"], b_["alpha_flat"])
    assert g1["lanes_per_row"] in (4, 8, 16, 32) and g1["block_threads"] in (256, 512, 1024)
    for lpr, thr in ((4, 256), (16, 1024)):
        f = S.spar_sink_batched(sets, pairs, s, lanes_per_row=lpr, block_threads=thr, **kw)
        assert (f["lanes_per_row"], f["block_threads"]) == (lpr, thr)
        for p in range(len(pairs)):
            assert abs(f["results"][p]["iters"] - r["results"][p]["iters"]) <= 2
            assert abs(f["results"][p]["obj"] - r["results"][p]["obj"]) <= 2e-6 * abs(r["results"][p]["obj"])


def test_batch_bf16_values(S, uot_batch):
    sets, pairs, s, kw, r = uot_batch
    h = S.spar_sink_batched(sets, pairs, s, kdtype="bf16", **kw)
    for p in range(len(pairs)):
        rel = abs(h["results"][p]["obj"] - r["results"][p]["obj"]) / abs(r["results"][p]["obj"])
        assert rel < 2.0 ** -7, (p, rel)


@pytest.fixture(scope="module")
def uot_batch_skip(S):
    sets = _sets(5, [420, 650, 300, 520, 800])
    pairs = _pairs(5)
    s = [12.0 * math.sqrt(len(sets[i][1]) * len(sets[j][1])) * math.log(len(sets[i][1])) for i, j in pairs]
    kw = dict(eps=0.01, lam=1.0, tol=1e-5, max_iter=5000, seed=77, problem_id=3,
              cost_norm=S.COST_SCALE, cost_scale=SCALE)
    r = S.spar_sink_batched(sets, pairs, s, sampler="skip", **kw)
    return sets, pairs, s, kw, r


def test_batch_skip_counts_follow_the_oracle_stream(S, orc, uot_batch_skip):
    """Skip sampler in the batch: every pair draws the stream of a single problem
    with id problem_id + p, so its sketch count equals the oracle's skip count."""
    sets, pairs, s, kw, r = uot_batch_skip
    assert r["status_code"] == 0
    for p, (i, j) in enumerate(pairs):
        (x, a), (y, b) = sets[i], sets[j]
        P = orc.OracleProblem(a, b, kw["eps"], s[p], 1.0, x=x, y=y, seed=kw["seed"], pid=kw["problem_id"] + p,
                              cost_norm=S.COST_SCALE, cost_scale=SCALE)
        _, nnz = P.skip_count()
        assert r["results"][p]["nnz"] == nnz, p


def test_batch_skip_pairs_equal_single_skip_solves(S, uot_batch_skip):
    sets, pairs, s, kw, r = uot_batch_skip
    for p, (i, j) in enumerate(pairs):
        (x, a), (y, b) = sets[i], sets[j]
        g = S.spar_sink_uot(a, b, x, y, eps=kw["eps"], lam=1.0, s=s[p], tol=kw["tol"], max_iter=5000, dtype="f32",
                            seed=kw["seed"], problem_id=kw["problem_id"] + p, cost_norm=S.COST_SCALE,
                            cost_scale=SCALE, log_domain=1, sampler="skip")
        rb = r["results"][p]
        assert rb["status"] == 0 and rb["nnz"] == g["nnz"], p
        assert abs(rb["iters"] - g["iters"]) <= max(2, 0.03 * g["iters"]), (p, rb["iters"], g["iters"])
        assert abs(rb["obj"] - g["obj"]) <= 2e-6 * abs(g["obj"]), p
        assert torch.allclose(r["alpha"][p], g["alpha"], rtol=0, atol=2e-5)


def test_batch_skip_matches_oracle(S, orc, uot_batch_skip):
    sets, pairs, s, kw, r = uot_batch_skip
    for p in (0, 5, 9):
        i, j = pairs[p]
        (x, a), (y, b) = sets[i], sets[j]
        P = orc.OracleProblem(a, b, kw["eps"], s[p], 1.0, x=x, y=y, seed=kw["seed"], pid=kw["problem_id"] + p,
                              cost_norm=S.COST_SCALE, cost_scale=SCALE)
        sk = P.sparsify(sampler="skip")
        o = orc.spar_sink(P, tol=kw["tol"], max_iter=5000, log_domain=True, sketch=sk)
        rb = r["results"][p]
        assert rb["nnz"] == sk["nnz"], p
        assert abs(rb["iters"] - o["info"]["iters"]) <= max(3, 0.05 * o["info"]["iters"]), p
        assert abs(rb["obj"] - o["obj"]) <= 1e-5 * abs(o["obj"]), p


def test_batch_skip_ot_matches_oracle(S, orc):
    sets = [(x, (w / w.sum()).astype(np.float32).astype(np.float64)) for x, w in _sets(6, [350, 500, 610])]
    pairs = [(0, 1), (1, 2), (2, 0), (1, 1)]
    s = [8000.0, 12000.0, 9000.0, 15000.0]
    r = S.spar_sink_batched(sets, pairs, s, eps=0.02, tol=1e-5, max_iter=5000, seed=5, cost_norm=S.COST_MAXNORM,
                            sampler="skip")
    assert r["status_code"] == 0
    for p, (i, j) in enumerate(pairs):
        (x, a), (y, b) = sets[i], sets[j]
        P = orc.OracleProblem(a, b, 0.02, s[p], math.inf, x=x, y=y, seed=5, pid=p)
        sk = P.sparsify(sampler="skip")
        o = orc.spar_sink(P, tol=1e-5, max_iter=5000, log_domain=True, sketch=sk)
        rb = r["results"][p]
        assert rb["nnz"] == sk["nnz"], p
        assert abs(rb["obj"] - o["obj"]) <= 1e-5 * abs(o["obj"]) + 1e-7, (p, rb["obj"], o["obj"])


def test_batch_graph_follows_the_sampler(S, uot_batch, uot_batch_skip):
    """A captured batch keyed by its parameters: the same workspace replayed with
    the other sampler runs that sampler's sketch."""
    sets, pairs, s, kw, r_el = uot_batch
    _, _, _, _, r_sk = uot_batch_skip
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        g1 = S.spar_sink_batched(sets, pairs, s, use_graph=1, **kw)
        g2 = S.spar_sink_batched(sets, pairs, s, use_graph=1, sampler="skip", workspace=g1["workspace"], **kw)
        g3 = S.spar_sink_batched(sets, pairs, s, use_graph=1, workspace=g1["workspace"], **kw)
    torch.cuda.synchronize()
    for p in range(len(pairs)):
        assert g1["results"][p]["nnz"] == g3["results"][p]["nnz"] == r_el["results"][p]["nnz"], p
        assert g2["results"][p]["nnz"] == r_sk["results"][p]["nnz"], p
