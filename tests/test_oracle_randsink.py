"""Pins for the oracle's equal-probability sampler (the Rand-Sink control of
section 5: Eq. (pois) with p_ij = 1/(n m) for every element, whatever the
weights, the cost or lambda).

- every kept element carries p* = min(1, s / (n m)) up to binary32 rounding;
- per-element inclusion frequencies over many Philox problem ids against that
  p*, for the element sampler and the skip sampler (whose row bound then
  equals p*, so every candidate is accepted), and E[nnz] = n m p*;
- a budget of 2 n m keeps every element: Spar-Sink then is Sinkhorn;
- on the WFR UOT problem of the section 5 simulations (total masses 5 and 3,
  eps = lambda = 0.1, eta for about half of K non-zero), the paper's
  probabilities (Eq. pij-uot) give a much smaller error than equal ones at
  the same budget, and their error falls as s grows.
"""
import math

import numpy as np
import pytest
from scipy import stats

from paper_2306_06581_gb300 import inputs


def _equal_pstar(n, m, s):
    return min(1.0, s / (n * m))


@pytest.mark.parametrize("lam,kind", [(math.inf, "sqeuclid"), (1.0, "sqeuclid"), (0.5, "wfr")])
def test_every_kept_element_has_the_equal_probability(orc, lam, kind):
    w = inputs.small_problem(n=40, m=55, d=2, seed=3)
    s = 300.0
    extra = dict(cost_kind="wfr", eta=0.5, cost_norm=0) if kind == "wfr" else {}
    P = orc.OracleProblem(w.a, w.b, 0.1, s, lam, x=w.x, y=w.y, probs="uniform", **extra)
    p = _equal_pstar(40, 55, s)
    for sampler in ("element", "skip"):
        sk = P.sparsify(sampler=sampler)
        assert sk["nnz"] > 0
        ps = sk["pstar"].astype(np.float64)
        assert np.all(ps == ps[0])
        assert abs(ps[0] - p) <= 2.5e-7 * p      # two binary32 roundings


@pytest.fixture(scope="module")
def freq(orc):
    w = inputs.small_problem(n=5, m=36, d=2, seed=9, lam=1.0)
    s, R = 54.0, 2000                  # p* = 0.3
    n, m = 5, 36
    out = {}
    for sampler in ("element", "skip"):
        hits = np.zeros((n, m))
        nnz = np.zeros(R)
        for pid in range(R):
            P = orc.OracleProblem(w.a, w.b, 0.1, s, 1.0, x=w.x, y=w.y, pid=pid, probs="uniform")
            sk = P.sparsify(sampler=sampler)
            rows = np.repeat(np.arange(n), np.diff(sk["row_ptr"]))
            hits[rows, sk["col_idx"]] += 1
            nnz[pid] = sk["nnz"]
        out[sampler] = (hits / R, nnz)
    return n, m, s, R, out


@pytest.mark.parametrize("sampler", ["element", "skip"])
def test_inclusion_frequencies_and_count(freq, sampler):
    n, m, s, R, out = freq
    f, nnz = out[sampler]
    p = _equal_pstar(n, m, s)
    z = (f - p) / math.sqrt(p * (1 - p) / R)
    assert np.abs(z).max() < 5.0, np.abs(z).max()
    sd = math.sqrt(n * m * p * (1 - p) / R)
    assert abs(nnz.mean() - n * m * p) < 5 * sd


@pytest.mark.parametrize("lam", [math.inf, 1.0])
def test_full_budget_is_sinkhorn(orc, lam):
    w = inputs.small_problem(n=20, m=24, d=3, seed=5, mass_b=1.0 if math.isinf(lam) else 1.4)
    P = orc.OracleProblem(w.a, w.b, 0.2, 2 * 20 * 24, lam, x=w.x, y=w.y, probs="uniform")
    sk = P.sparsify()
    assert sk["nnz"] == 20 * 24 and np.all(sk["pstar"] == 1.0)
    sp = orc.spar_sink(P, tol=1e-12, max_iter=100000, sketch=sk)
    de = orc.dense_sinkhorn(P, tol=1e-12, max_iter=100000)
    assert sp["obj"] == pytest.approx(de["obj"], rel=1e-12)


def _wfr_uot_case(n, d, seed):
    """Support x_i ~ U(0,1)^d shared by both measures; a and b follow N(1/3, 1/20)
    and N(1/2, 1/20) densities over the grid i/n, with total masses 5 and 3;
    eta puts the median distance at pi eta, so about half of K is non-zero."""
    rng = np.random.default_rng(seed)
    x = rng.uniform(0, 1, (n, d))
    g = (np.arange(n) + 0.5) / n
    a = stats.norm.pdf(g, 1 / 3, math.sqrt(1 / 20))
    b = stats.norm.pdf(g, 1 / 2, math.sqrt(1 / 20))
    a, b = 5 * a / a.sum(), 3 * b / b.sum()
    dist = np.sqrt(((x[:, None] - x[None]) ** 2).sum(-1))
    return x, a, b, float(np.quantile(dist, 0.5)) / math.pi


def test_paper_probabilities_beat_equal_ones_on_wfr_uot(orc):
    n, d, eps, lam = 300, 5, 0.1, 0.1
    x, a, b, eta = _wfr_uot_case(n, d, 1)
    kw = dict(x=x, y=x, cost_norm=0, cost_kind="wfr", eta=eta)
    K, _ = orc.OracleProblem(a, b, eps, 1.0, lam, **kw).dense_kernel()
    assert 0.4 < (K > 0).mean() < 0.6
    ref = orc.dense_sinkhorn(orc.OracleProblem(a, b, eps, 1.0, lam, **kw), tol=1e-9, max_iter=20000)["obj"]
    s0 = inputs.s0(n)
    err = {}
    for probs in ("paper", "uniform"):
        for f in (4.0, 16.0):
            e = []
            for pid in range(12):
                P = orc.OracleProblem(a, b, eps, f * s0, lam, pid=pid, probs=probs, **kw)
                r = orc.spar_sink(P, tol=1e-9, max_iter=20000)
                e.append(abs(r["obj_sparse"] - ref) / abs(ref))
            err[probs, f] = float(np.mean(e))
    for f in (4.0, 16.0):
        assert err["paper", f] < 0.2 * err["uniform", f], err
    assert err["paper", 16.0] < 0.5 * err["paper", 4.0], err
