"""Pins for the IBP / Spar-IBP oracle (fixed-support Wasserstein
barycenters, the paper's appendix on barycenters).

- one measure: the fixed point has u = 1, so q* = K (b / K^T 1) in closed form;
  identical measures give the same barycenter whatever the weights;
- the fixed point of several measures satisfies every plan's marginals:
  u_k * (K_k v_k) = q and v_k * (K_k^T u_k) = b_k;
- the barycenter minimises sum_k w_k OT_eps(q, b_k), each OT_eps computed
  from its definition by a converged Sinkhorn, checked by a generic optimiser
  over the simplex on a tiny instance;
- Spar-IBP with p* = 1 everywhere is IBP; its error against IBP falls as the
  budget s grows.
"""
import math

import numpy as np
import pytest
from scipy import optimize, stats


def _measures(n, seed=0):
    """The paper's synthetic recipe on a 1-D grid i/n: a Gaussian, a two-component
    mixture and a t_5 density, each plus 1e-2 of its maximum, normalised."""
    g = (np.arange(n) + 0.5) / n
    b1 = stats.norm.pdf(g, 0.2, math.sqrt(1 / 50))
    b2 = 0.5 * stats.norm.pdf(g, 0.5, math.sqrt(1 / 60)) + 0.5 * stats.norm.pdf(g, 0.8, math.sqrt(1 / 80))
    b3 = stats.t.pdf((g - 0.6) / math.sqrt(1 / 100), 5)
    out = []
    for b in (b1, b2, b3):
        b = b + 1e-2 * b.max()
        out.append(b / b.sum())
    return out


@pytest.fixture(scope="module")
def ibpo(orc):
    from oracle import ibp_oracle
    return ibp_oracle


def _support(n, d, seed):
    return np.random.default_rng(seed).uniform(0, 1, (n, d))


def test_single_measure_closed_form(ibpo):
    x = _support(40, 3, 1)
    b = _measures(40)[1]
    K = ibpo.dense_kernels(x, [b], 0.1)[0]
    q, info = ibpo.ibp([K], [b], [1.0], tol=1e-13)
    q_closed = K @ (b / (K.T @ np.ones(40)))
    assert np.allclose(q, q_closed, rtol=1e-9, atol=1e-15)
    # identical measures: the same barycenter for any weights
    q3, _ = ibpo.ibp([K, K, K], [b, b, b], [0.2, 0.5, 0.3], tol=1e-13)
    assert np.allclose(q3, q_closed, rtol=1e-9, atol=1e-15)


def test_fixed_point_marginals(ibpo):
    n = 50
    x = _support(n, 2, 2)
    bs = _measures(n)
    Ks = ibpo.dense_kernels(x, bs, 0.05)
    q, info = ibpo.ibp(Ks, bs, [1 / 3] * 3, tol=1e-12, max_iter=50000)
    assert info["delta"] <= 1e-12
    for k in range(3):
        u, v = info["u"][k], info["v"][k]
        assert np.allclose(v * (Ks[k].T @ u), bs[k], rtol=1e-9, atol=1e-14)
        assert np.allclose(u * (Ks[k] @ v), q, rtol=1e-7, atol=1e-12)
    assert abs(q.sum() - 1.0) < 1e-8


def test_fixed_point_marginals_rectangular(ibpo, orc):
    # measures on their own supports (n_k != n): K_k is n x n_k and not symmetric
    n, eps = 30, 0.1
    x = _support(n, 2, 12)
    rng = np.random.default_rng(13)
    Ks, bs = [], []
    for k, nk in enumerate((40, 25, 35)):
        y = _support(nk, 2, 20 + k) * 0.8 + 0.1
        b = rng.uniform(0.2, 1.0, nk)
        b /= b.sum()
        K, _ = orc.OracleProblem(np.full(n, 1.0 / n), b, eps, 1.0, math.inf, x=x, y=y).dense_kernel()
        Ks.append(K)
        bs.append(b)
    q, info = ibpo.ibp(Ks, bs, [0.5, 0.2, 0.3], tol=1e-12, max_iter=100000)
    assert info["delta"] <= 1e-12
    for k in range(3):
        u, v = info["u"][k], info["v"][k]
        assert np.allclose(v * (Ks[k].T @ u), bs[k], rtol=1e-9, atol=1e-14)
        assert np.allclose(u * (Ks[k] @ v), q, rtol=1e-7, atol=1e-12)


def _ot_eps(q, b, C, eps):
    """OT_eps(q, b) = min <T, C> - eps H(T), H(T) = -sum T (log T - 1), by Sinkhorn
    iterations in log form run to convergence (the definition, written out)."""
    f = np.zeros(len(q))
    g = np.zeros(len(b))
    lq, lb = np.log(q), np.log(b)
    for _ in range(20000):
        f_old = f
        f = eps * lq - eps * np.logaddexp.reduce((g[None, :] - C) / eps, axis=1)
        g = eps * lb - eps * np.logaddexp.reduce((f[:, None] - C) / eps, axis=0)
        if np.abs(f - f_old).max() < 1e-13:
            break
    T = np.exp((f[:, None] + g[None, :] - C) / eps)
    return float((T * C).sum() + eps * (T * (np.log(T) - 1)).sum())


def test_barycenter_minimises_weighted_entropic_cost(ibpo):
    n, eps = 5, 0.2
    x = _support(n, 2, 3)
    rng = np.random.default_rng(4)
    bs = [rng.uniform(0.2, 1.0, n) for _ in range(2)]
    bs = [b / b.sum() for b in bs]
    w = np.array([0.35, 0.65])
    Ks = ibpo.dense_kernels(x, bs, eps)
    C = -eps * np.log(Ks[0])
    q, _ = ibpo.ibp(Ks, bs, w, tol=1e-14, max_iter=200000)

    def obj(z):
        qq = np.exp(z - z.max())
        qq = qq / qq.sum()
        return sum(w[k] * _ot_eps(qq, bs[k], C, eps) for k in range(2))

    z0 = np.log(np.full(n, 1.0 / n))
    res = optimize.minimize(obj, z0, method="Nelder-Mead",
                            options={"xatol": 1e-10, "fatol": 1e-14, "maxiter": 40000, "maxfev": 40000})
    qm = np.exp(res.x - res.x.max())
    qm /= qm.sum()
    assert np.abs(qm - q).sum() < 2e-4, (qm, q)
    assert obj(np.log(q)) <= res.fun + 1e-9


def test_spar_ibp_probabilities(ibpo):
    # the appendix's p_{k,ij} = sqrt(b_{k,j}) / (n sum_j sqrt(b_{k,j})) (equal within a column)
    n, s = 60, 400.0
    x = _support(n, 2, 7)
    bs = _measures(n)
    _, sks = ibpo.spar_ibp_sketches(x, bs, 0.1, s)
    for b, sk in zip(bs, sks):
        p = np.minimum(1.0, s * np.sqrt(b) / (n * np.sqrt(b).sum()))
        assert np.allclose(sk["pstar"], p[sk["col_idx"]], rtol=1e-6, atol=0)


def test_spar_ibp_full_budget_is_ibp(ibpo):
    n = 30
    x = _support(n, 3, 5)
    bs = _measures(n)
    Ks = ibpo.dense_kernels(x, bs, 0.1)
    q, _ = ibpo.ibp(Ks, bs, [1 / 3] * 3, tol=1e-12)
    qs, _ = ibpo.spar_ibp(x, bs, [1 / 3] * 3, 0.1, s=1e9, tol=1e-12)   # every p* clipped to 1
    assert np.allclose(qs, q, rtol=1e-10, atol=1e-15)


def test_spar_ibp_error_falls_with_budget(ibpo):
    # s / s0(n) = 10 and 60 at n = 200 keep 4% and 24% of the elements
    n, eps = 200, 0.1
    x = _support(n, 5, 6)
    bs = _measures(n)
    w = [1 / 3] * 3
    Ks = ibpo.dense_kernels(x, bs, eps)
    q, _ = ibpo.ibp(Ks, bs, w, tol=1e-10)
    s0 = 1e-3 * n * math.log(n) ** 4
    errs = []
    for f in (10.0, 60.0):
        e = []
        for seed in range(6):
            qs, _ = ibpo.spar_ibp(x, bs, w, eps, s=f * s0, tol=1e-10, seed=1000 + seed)
            e.append(np.abs(qs - q).sum())
        errs.append(np.mean(e))
    assert errs[1] < 0.6 * errs[0], errs
