"""Pins for the oracle's skip sampler (thinning by geometric skips over a row
bound): it must draw the law of Eq. (pois) with Eq. (pij-ot) or Eq. (pij-uot)
-- every element kept independently with probability p*_ij = min(1, s p_ij).

- the spec log(1 - q) against FP64 log1p;
- per-element inclusion frequencies over many Philox problem ids against
  p*_ij (binomial z-scores), including a row whose bound q_i reaches 1;
- pairwise independence of neighbouring elements (the gap process is where a
  wrong construction would correlate them);
- E[nnz] = sum p*;
- zero weights give empty rows and columns; p* = 1 everywhere gives the full
  matrix; the sketch's values are the definition K_ij / p*_ij.
"""
import math

import numpy as np
import pytest

from paper_2306_06581_gb300 import inputs


def _problem(orc, a, b, x, y, s, pid=0, seed=0x5EED):
    return orc.OracleProblem(a, b, 0.1, s, math.inf, x=x, y=y, seed=seed, pid=pid)


def _pstar(a, b, s):
    sa, sb = np.sqrt(a), np.sqrt(b)
    return np.minimum(1.0, s * np.outer(sa, sb) / (sa.sum() * sb.sum()))


def test_log1m_against_fp64(orc):
    q = np.concatenate([np.logspace(-9, math.log10(0.2499), 4000), np.linspace(0.25, 0.9999, 4000),
                        np.array([0.25, 0.5, 0.75, 2.0 ** -24, 1.0 - 2.0 ** -24])]).astype(np.float32)
    got = orc.log1m32(q).astype(np.float64)
    ref = np.log1p(-q.astype(np.float64))
    rel = np.abs(got - ref) / np.abs(ref)
    assert rel.max() < 6e-7, rel.max()   # a few binary32 ulps


def _freq(orc, a, b, x, y, s, K):
    n, m = a.size, b.size
    hits = np.zeros((n, m))
    both = np.zeros((n, m - 1))
    nnz = np.zeros(K)
    for pid in range(K):
        P = _problem(orc, a, b, x, y, s, pid=pid)
        ind = np.zeros((n, m))
        for i in range(n):
            ind[i, P.skip_row(i)["cols"]] = 1.0
        hits += ind
        both += ind[:, :-1] * ind[:, 1:]
        nnz[pid] = ind.sum()
    return hits / K, both / K, nnz


@pytest.fixture(scope="module")
def freq_case(orc):
    rng = np.random.default_rng(11)
    n, m = 4, 48
    a = rng.uniform(0.05, 1.0, n)
    a[3] = 40.0                       # a heavy row: its bound q reaches 1
    b = rng.uniform(0.0, 1.0, m)
    b[5] = 0.0                        # a column that can never be kept
    x = rng.standard_normal((n, 2))
    y = rng.standard_normal((m, 2))
    s = 60.0
    K = 2500
    f, f2, nnz = _freq(orc, a, b, x, y, s, K)
    return a, b, s, K, f, f2, nnz


def test_inclusion_frequencies(freq_case):
    a, b, s, K, f, _, _ = freq_case
    p = _pstar(a, b, s)
    assert p[3].max() == 1.0 and 0.0 < p[:3].max() < 1.0
    sd = np.sqrt(np.maximum(p * (1 - p), 1e-12) / K)
    z = (f - p) / sd
    inner = (p < 1) & (p * K >= 25)
    assert inner.sum() > 120
    assert np.abs(z[inner]).max() < 5.0, np.abs(z[inner]).max()
    small = (p > 0) & (p * K < 25)
    assert f[small].sum() * K == pytest.approx(p[small].sum() * K, abs=6 * math.sqrt(p[small].sum() * K + 1))
    assert np.all(f[p == 1.0] == 1.0)
    assert np.all(f[:, 5] == 0.0)


def test_neighbours_independent(freq_case):
    a, b, s, K, _, f2, _ = freq_case
    p = _pstar(a, b, s)
    pp = p[:, :-1] * p[:, 1:]
    sd = np.sqrt(np.maximum(pp * (1 - pp), 1e-12) / K)
    z = (f2 - pp) / sd
    inner = (pp < 1) & (pp * K >= 25)   # expected joint counts large enough for the normal law
    assert inner.sum() > 60
    assert np.abs(z[inner]).max() < 5.0, np.abs(z[inner]).max()


def test_expected_count(freq_case):
    a, b, s, K, _, _, nnz = freq_case
    p = _pstar(a, b, s)
    sd = math.sqrt((p * (1 - p)).sum() / K)
    assert abs(nnz.mean() - p.sum()) < 5 * sd


def test_zero_weight_row_and_full_matrix(orc):
    w = inputs.small_problem(n=12, m=15, d=2, seed=4)
    a = w.a.copy()
    a[2] = 0.0
    P = _problem(orc, a, w.b, w.x, w.y, w.s)
    assert P.skip_row(2)["cols"].size == 0
    Pf = _problem(orc, w.a, w.b, w.x, w.y, 1e9)   # every p* clipped to 1
    sk = Pf.sparsify(sampler="skip")
    assert sk["nnz"] == 12 * 15
    assert np.array_equal(np.diff(sk["row_ptr"]), np.full(12, 15))


def test_values_follow_definition(orc):
    w = inputs.small_problem(n=30, m=40, d=3, seed=6)
    P = _problem(orc, w.a, w.b, w.x, w.y, w.s)
    sk = P.sparsify(sampler="skip")
    rows = np.repeat(np.arange(30), np.diff(sk["row_ptr"]))
    D = ((w.x[rows] - w.y[sk["col_idx"]]) ** 2).sum(1)
    Dall = ((w.x[:, None, :] - w.y[None, :, :]) ** 2).sum(-1)
    C = D / Dall.astype(np.float32).max()
    ps = _pstar(w.a, w.b, w.s)[rows, sk["col_idx"]]
    assert np.allclose(sk["val"], np.exp(-C / 0.1) / ps, rtol=2e-6)
    assert np.allclose(sk["pstar"], ps, rtol=1e-6)
    # the skip stream is not the element stream (a different random source)
    el = P.sparsify()
    assert not (el["nnz"] == sk["nnz"] and np.array_equal(el["col_idx"], sk["col_idx"]))


def test_uot_inclusion_frequencies(orc):
    # Eq. (pij-uot): p_ij proportional to (a_i b_j)^gamma exp(-C_ij / (2 lam + eps))
    rng = np.random.default_rng(21)
    n, m, lam, eps = 3, 40, 1.0, 0.1
    a = rng.uniform(0.05, 1.0, n)
    b = rng.uniform(0.05, 1.5, m)
    x = rng.standard_normal((n, 2))
    y = rng.standard_normal((m, 2)) + 0.5
    s, K = 100.0, 2500   # s / Z > 1: a row bound without the factor s / Z would be too small
    D = ((x[:, None, :] - y[None, :, :]) ** 2).sum(-1)
    C = D / D.astype(np.float32).max()
    g = lam / (2 * lam + eps)
    w = np.outer(a, b) ** g * np.exp(-C / (2 * lam + eps))
    p = np.minimum(1.0, s * w / w.sum())
    hits = np.zeros((n, m))
    for pid in range(K):
        P = orc.OracleProblem(a, b, eps, s, lam, x=x, y=y, pid=pid)
        for i in range(n):
            hits[i, P.skip_row(i)["cols"]] += 1.0
    f = hits / K
    z = (f - p) / np.sqrt(np.maximum(p * (1 - p), 1e-12) / K)
    inner = (p < 1) & (p * K >= 25)
    assert inner.sum() > 60
    assert np.abs(z[inner]).max() < 5.0, np.abs(z[inner]).max()
    # the per-element and skip streams agree in expectation
    assert abs(f.sum() - p.sum()) < 5 * math.sqrt((p * (1 - p)).sum() / K)
