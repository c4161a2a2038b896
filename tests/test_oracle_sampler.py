"""Pins for the oracle's sampler: Eq. (pois) with Eq. (pij-ot) / (pij-uot).

- the binary32 decision probabilities agree with the FP64 definitions of
  Eq. (pij-ot) and Eq. (pij-uot) up to binary32 rounding;
- lambda -> infinity turns the UOT probabilities into the OT ones (sec. 3.3);
- unbiasedness E[K~] = K and E[nnz] = sum p* <= s (sec. 3.2), Monte Carlo
  over Philox seeds, and per-element inclusion frequencies (chi-square);
- p* = 1 everywhere makes K~ = K and Spar-Sink identical to Sinkhorn;
- the CSC is the stable transpose of the CSR.
"""
import math

import numpy as np
import pytest
from scipy import stats

from paper_2306_06581_gb300 import inputs


def _prob(orc, w, **kw):
    args = dict(x=w.x, y=w.y, seed=w.seed, pid=w.pid)
    args.update(kw)
    return orc.OracleProblem(w.a, w.b, kw.pop("eps", w.eps), kw.pop("s", w.s), kw.pop("lam", w.lam),
                             **{k: v for k, v in args.items() if k not in ("eps", "s", "lam")})


def _sqdist(x, y):
    return ((x[:, None, :] - y[None, :, :]) ** 2).sum(-1)


def test_ot_probability_matches_definition(orc):
    w = inputs.small_problem(n=40, m=50, d=3, seed=3)
    P = orc.OracleProblem(w.a, w.b, w.eps, w.s, math.inf, x=w.x, y=w.y)
    sq = np.sqrt(np.outer(w.a, w.b))
    p_def = w.s * sq / sq.sum()                           # s p_ij, Eq. (pij-ot)
    got = np.array([[P.pstar_raw(i, j) for j in range(w.m)] for i in range(w.n)], np.float64)
    assert np.allclose(got, p_def, rtol=6e-7, atol=0)


@pytest.mark.parametrize("lam,eps", [(1.0, 0.05), (0.1, 0.1), (5.0, 0.01)])
def test_uot_probability_matches_definition(orc, lam, eps):
    w = inputs.small_problem(n=30, m=35, d=4, seed=4, mass_b=1.5)
    P = orc.OracleProblem(w.a, w.b, eps, w.s, lam, x=w.x, y=w.y)
    C = _sqdist(w.x, w.y)
    C = C / C.max()
    K = np.exp(-C / eps)
    g = lam / (2 * lam + eps)
    num = np.outer(w.a, w.b) ** g * K ** (eps / (2 * lam + eps))   # Eq. (pij-uot) numerator
    p_def = w.s * num / num.sum()
    got = np.array([[P.pstar_raw(i, j) for j in range(w.m)] for i in range(w.n)], np.float64)
    assert np.allclose(got, p_def, rtol=3e-6, atol=0)


def test_uot_probability_tends_to_ot(orc):
    w = inputs.small_problem(n=25, m=25, d=2, seed=5)
    Pot = orc.OracleProblem(w.a, w.b, 0.1, w.s, math.inf, x=w.x, y=w.y)
    Puot = orc.OracleProblem(w.a, w.b, 0.1, w.s, 1e7, x=w.x, y=w.y)
    for i, j in [(0, 0), (3, 7), (24, 24), (11, 2)]:
        assert abs(Puot.pstar_raw(i, j) / Pot.pstar_raw(i, j) - 1) < 1e-5


def test_inclusion_rate_over_many_decisions(orc):
    # one sketch of 4.2e6 decisions: the kept count is a sum of independent
    # Bernoulli(p*) (sd ~ 1e3), so a 1% bias in the keep rule shows at ~10 sd;
    # p* from the FP64 definitions (within ~1e-6 of the binary32 spec)
    n, m = 2000, 2100
    for lam in (math.inf, 1.0):
        w = inputs.small_problem(n=n, m=m, d=3, seed=17, mass_b=1.0 if math.isinf(lam) else 1.5)
        s = 0.3 * n * m
        eps = 0.1
        P = orc.OracleProblem(w.a, w.b, eps, s, lam, x=w.x, y=w.y, seed=77)
        _, nnz = P.count()
        if math.isinf(lam):
            q = np.outer(np.sqrt(w.a), np.sqrt(w.b))
        else:
            x32, y32 = w.x.astype(np.float32).astype(np.float64), w.y.astype(np.float32).astype(np.float64)
            D = ((x32[:, None, :] - y32[None, :, :]) ** 2).sum(-1)
            g = lam / (2 * lam + eps)
            q = np.outer(w.a, w.b) ** g * np.exp(-(D / D.max()) / (2 * lam + eps))
        p = np.minimum(1.0, s * q / q.sum())
        sd = math.sqrt((p * (1 - p)).sum())
        assert abs(nnz - p.sum()) < 5 * sd + 1e-5 * p.sum(), (lam, nnz, p.sum(), sd)


def test_unbiased_and_expected_nnz(orc):
    n, m = 10, 12
    w = inputs.small_problem(n=n, m=m, d=2, seed=6, eps=0.5)
    s = 40.0
    K, _ = orc.OracleProblem(w.a, w.b, w.eps, s, math.inf, x=w.x, y=w.y).dense_kernel()
    R = 3000
    acc = np.zeros((n, m))
    inc = np.zeros((n, m))
    nnz = []
    for r in range(R):
        P = orc.OracleProblem(w.a, w.b, w.eps, s, math.inf, x=w.x, y=w.y, seed=1000 + r)
        sk = P.sparsify()
        rows = np.repeat(np.arange(n), np.diff(sk["row_ptr"]))
        acc[rows, sk["col_idx"]] += sk["val"]
        inc[rows, sk["col_idx"]] += 1
        nnz.append(sk["nnz"])
    P0 = orc.OracleProblem(w.a, w.b, w.eps, s, math.inf, x=w.x, y=w.y)
    pst = np.array([[min(1.0, P0.pstar_raw(i, j)) for j in range(m)] for i in range(n)])
    # E[nnz] = sum p* <= s
    assert pst.sum() <= s * (1 + 1e-6)
    sd_nnz = math.sqrt((pst * (1 - pst)).sum() / R)
    assert abs(np.mean(nnz) - pst.sum()) < 5 * sd_nnz
    # E[K~] = K, with Var K~_ij = K^2 (1/p* - 1)
    mean = acc / R
    sd = K * np.sqrt((1 / pst - 1) / R)
    z = np.abs(mean - K) / np.where(sd > 0, sd, 1)
    assert z.max() < 5.0
    # inclusion frequencies: chi-square against p*
    exp_inc = R * pst
    mask = (pst > 0) & (pst < 1)
    chi2 = (((inc - exp_inc) ** 2) / (exp_inc * (1 - pst)))[mask].sum()
    assert chi2 < stats.chi2.ppf(0.9999, mask.sum())


def test_all_included_reduces_to_sinkhorn(orc):
    w = inputs.small_problem(n=30, m=20, d=3, seed=7, eps=0.2)
    P = orc.OracleProblem(w.a, w.b, w.eps, 1e9, math.inf, x=w.x, y=w.y)
    sk = P.sparsify()
    assert sk["nnz"] == 30 * 20 and (sk["pstar"] == 1.0).all()
    K, _ = P.dense_kernel()
    assert np.array_equal(sk["val"].reshape(30, 20), K)
    sp = orc.spar_sink(P, tol=1e-10, max_iter=2000, sketch=sk)
    de = orc.dense_sinkhorn(P, tol=1e-10, max_iter=2000)
    assert sp["info"]["iters"] == de["info"]["iters"]
    assert np.allclose(sp["alpha"], de["alpha"], rtol=0, atol=1e-12)
    assert abs(sp["obj"] - de["obj"]) < 1e-12
    assert sp["obj"] == sp["obj_sparse"]


def test_csc_is_stable_transpose(orc):
    w = inputs.small_problem(n=70, m=90, d=3, seed=8)
    sk = orc.OracleProblem(w.a, w.b, w.eps, 2000.0, math.inf, x=w.x, y=w.y).sparsify()
    n, m = 70, 90
    D = np.zeros((n, m))
    rows = np.repeat(np.arange(n), np.diff(sk["row_ptr"]))
    D[rows, sk["col_idx"]] = sk["val"]
    DT = np.zeros((n, m))
    cols = np.repeat(np.arange(m), np.diff(sk["col_ptr"]))
    DT[sk["row_idx"], cols] = sk["valT"]
    assert np.array_equal(D, DT)
    for j in range(m):
        seg = sk["row_idx"][sk["col_ptr"][j]:sk["col_ptr"][j + 1]]
        assert (np.diff(seg) > 0).all()
    for i in range(n):
        seg = sk["col_idx"][sk["row_ptr"][i]:sk["row_ptr"][i + 1]]
        assert (np.diff(seg) > 0).all()
    assert np.array_equal(sk["val"][sk["perm"]], sk["valT"])


def test_values_and_log_values(orc):
    w = inputs.small_problem(n=50, m=40, d=5, seed=9, eps=0.05)
    P = orc.OracleProblem(w.a, w.b, w.eps, 300.0, math.inf, x=w.x, y=w.y)
    sk = P.sparsify()
    C = _sqdist(w.x, w.y)
    C = C / C.max()
    rows = np.repeat(np.arange(50), np.diff(sk["row_ptr"]))
    Cs = C[rows, sk["col_idx"]]
    # the divisor is the max of the binary32 distances: within binary32 rounding of the FP64 max
    assert np.allclose(sk["cost"], Cs, rtol=2e-7, atol=1e-15)
    Cx = sk["cost"]
    assert np.allclose(sk["val"], np.exp(-Cx / w.eps) / sk["pstar"], rtol=1e-13)
    assert np.allclose(sk["logval"], -Cx / w.eps - np.log(sk["pstar"].astype(np.float64)), rtol=1e-13)
    # the cost at the sampled elements is the raw distance over one common divisor
    D = ((w.x[:, None, :] - w.y[None]) ** 2).sum(-1)[rows, sk["col_idx"]]
    ratio = D / Cx
    assert np.allclose(ratio, ratio[0], rtol=1e-13)


def test_pattern_deterministic_and_stream_specific(orc):
    w = inputs.small_problem(n=60, m=60, d=3, seed=10)
    a = orc.OracleProblem(w.a, w.b, w.eps, 500.0, math.inf, x=w.x, y=w.y, seed=11).sparsify()
    b = orc.OracleProblem(w.a, w.b, w.eps, 500.0, math.inf, x=w.x, y=w.y, seed=11).sparsify()
    c = orc.OracleProblem(w.a, w.b, w.eps, 500.0, math.inf, x=w.x, y=w.y, seed=11, pid=1).sparsify()
    assert np.array_equal(a["col_idx"], b["col_idx"]) and np.array_equal(a["row_ptr"], b["row_ptr"])
    assert not (a["nnz"] == c["nnz"] and np.array_equal(a["col_idx"], c["col_idx"]))


def test_dense_cost_input_equals_points(orc):
    w = inputs.small_problem(n=20, m=25, d=3, seed=12)
    C = _sqdist(w.x, w.y)
    for lam in [math.inf, 1.0]:
        a = orc.OracleProblem(w.a, w.b, 0.1, 200.0, lam, x=w.x, y=w.y).sparsify()
        b = orc.OracleProblem(w.a, w.b, 0.1, 200.0, lam, C_=C).sparsify()
        # the decision cost is binary32 in both forms; the dense form rounds the FP64 cost,
        # the point form accumulates in binary32, so patterns may differ on rare ties only
        assert abs(a["nnz"] - b["nnz"]) <= 2
        assert np.allclose(a["val"][:5], b["val"][:5], rtol=1e-12) or a["nnz"] != b["nnz"]


@pytest.mark.parametrize("lam,kind", [(math.inf, "sqeuclid"), (1.0, "sqeuclid"), (0.5, "wfr"), (1.0, "uniform")])
def test_row_samplers_equal_full_sketch(orc, lam, kind):
    # The full-size GPU checks compare sampled rows with the oracle's per-row
    # samplers (every decision of a row re-derived from its counters): each
    # must reproduce its row of the full sketch exactly, for both samplers.
    w = inputs.small_problem(n=90, m=110, d=3, seed=31)
    kw = dict(x=w.x, y=w.y, seed=77, pid=2)
    if kind == "wfr":
        kw.update(cost_kind="wfr", eta=0.6, cost_norm=0)
    if kind == "uniform":
        kw.update(probs="uniform")
    P = orc.OracleProblem(w.a, w.b * (1.0 if math.isinf(lam) else 1.5), 0.1, 1500.0, lam, **kw)
    for sampler, row_fn, count_fn in (("element", P.sample_row, P.count), ("skip", P.skip_row, P.skip_count)):
        sk = P.sparsify(sampler=sampler)
        cnt, nnz = count_fn()
        assert nnz == sk["nnz"] and np.array_equal(cnt, np.diff(sk["row_ptr"]))
        assert sk["nnz"] > 0
        for i in range(P.n):
            lo, hi = sk["row_ptr"][i], sk["row_ptr"][i + 1]
            r = row_fn(i)
            assert np.array_equal(r["cols"], sk["col_idx"][lo:hi]), (sampler, i)
            for key, skey in (("val", "val"), ("logval", "logval"), ("pstar", "pstar"), ("cost", "cost")):
                assert np.array_equal(r[key], sk[skey][lo:hi]), (sampler, i, key)
