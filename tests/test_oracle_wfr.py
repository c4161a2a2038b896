"""Pins for the oracle's Wasserstein-Fisher-Rao cost (section 2.2):
C_ij = -log cos_+^2(d_ij / (2 eta)), d_ij the Euclidean distance, with
UOT sampling probabilities from Eq. (pij-uot).

- the binary32 spec cos against FP64 cos on [0, pi/2];
- transport is blocked exactly where d_ij >= pi eta: K_ij = 0 there, p* = 0,
  and no sketch ever holds such a pair;
- the decision probabilities against their FP64 definition;
- small angles: -log cos^2 z = z^2 + z^4/3 + ..., so with eta large the WFR
  solve approaches the squared-Euclidean solve with cost scale 4 eta^2, the
  gap shrinking like eta^-2;
- E[K~] = K by Monte Carlo over problem ids.
"""
import math

import numpy as np
import pytest


def _pts(n, d, seed, spread=1.0):
    return np.random.default_rng(seed).uniform(0, spread, (n, d))


def test_cos_spec(orc):
    z = np.linspace(0.0, math.pi / 2, 20001).astype(np.float32)
    got = orc.cos32(z).astype(np.float64)
    ref = np.cos(z.astype(np.float64))
    assert np.abs(got - ref).max() < 2.5e-7
    inner = z < 1.4
    assert (np.abs(got - ref)[inner] / ref[inner]).max() < 1e-6


def _wfr_problem(orc, n, m, eta, lam=1.0, eps=0.1, s=None, pid=0, seed=3):
    rng = np.random.default_rng(seed)
    x, y = _pts(n, 2, seed), _pts(m, 2, seed + 1)
    a = rng.uniform(0.2, 1.0, n)
    b = rng.uniform(0.2, 1.0, m)
    a, b = a / a.sum() * 1.2, b / b.sum() * 0.8
    s = s if s is not None else 0.3 * n * m
    P = orc.OracleProblem(a, b, eps, s, lam, x=x, y=y, cost_norm=0, cost_kind="wfr", eta=eta, pid=pid)
    return P, x, y, a, b


def test_blocked_transport(orc):
    eta = 0.12                          # pi eta = 0.377: a part of the unit square's pairs is blocked
    P, x, y, a, b = _wfr_problem(orc, 40, 50, eta)
    d = np.sqrt(((x[:, None, :] - y[None, :, :]) ** 2).sum(-1))
    K, Cn = P.dense_kernel()
    blocked = d >= math.pi * eta
    assert 0.2 < blocked.mean() < 0.9
    assert np.all(K[blocked] == 0.0) and np.all(np.isinf(Cn[blocked]))
    assert np.all(K[~blocked] > 0.0)
    sk = P.sparsify()
    rows = np.repeat(np.arange(40), np.diff(sk["row_ptr"]))
    assert sk["nnz"] > 0
    assert np.all(d[rows, sk["col_idx"]] < math.pi * eta)
    ps = np.array([[P.pstar_raw(i, j) for j in range(50)] for i in range(40)])
    assert np.all(ps[d >= math.pi * eta * (1 + 1e-6)] == 0.0)


def test_probability_matches_definition(orc):
    eta, lam, eps = 0.3, 1.0, 0.1
    P, x, y, a, b = _wfr_problem(orc, 30, 35, eta, lam, eps, s=200.0)
    d = np.sqrt(((x[:, None, :] - y[None, :, :]) ** 2).sum(-1))
    z = np.minimum(d / (2 * eta), math.pi / 2)
    g = lam / (2 * lam + eps)
    w = np.outer(a, b) ** g * np.cos(z) ** (2.0 / (2 * lam + eps))   # K^{eps/(2lam+eps)}
    p_def = 200.0 * w / w.sum()
    got = np.array([[P.pstar_raw(i, j) for j in range(35)] for i in range(30)], np.float64)
    ok = z < 1.3
    assert np.allclose(got[ok], p_def[ok], rtol=5e-6, atol=0)


def _dense_obj(orc, P):
    return orc.dense_sinkhorn(P, tol=1e-11, max_iter=200000)["obj"]


def test_small_angle_limit(orc):
    rng = np.random.default_rng(9)
    n, m = 25, 30
    x, y = _pts(n, 2, 11), _pts(m, 2, 12)
    a = rng.uniform(0.2, 1.0, n)
    b = rng.uniform(0.2, 1.0, m)
    a, b = a / a.sum(), b / b.sum() * 1.3
    dmax = math.sqrt(((x[:, None, :] - y[None, :, :]) ** 2).sum(-1).max())
    gaps = []
    for zmax in (0.08, 0.04):
        eta = dmax / (2 * zmax)
        # eps and lam follow the cost scale z^2, so the squared-Euclidean problem is the same at
        # both eta and the gap is the z^4 / 3 term of the cost alone
        eps, lam = 0.05 * zmax ** 2, zmax ** 2
        W = orc.OracleProblem(a, b, eps, 1.0, lam, x=x, y=y, cost_norm=0, cost_kind="wfr", eta=eta)
        Q = orc.OracleProblem(a, b, eps, 1.0, lam, x=x, y=y, cost_norm=2, cost_scale=4 * eta * eta)
        ow, oq = _dense_obj(orc, W), _dense_obj(orc, Q)
        gaps.append(abs(ow - oq) / abs(oq))
    assert gaps[0] < 1e-2
    assert 0.12 < gaps[1] / gaps[0] < 0.4, gaps     # z^4 / 3 relative to z^2: halving z quarters the gap


def test_unbiased_kernel(orc):
    eta = 0.25
    K = None
    acc = None
    R = 1500
    for pid in range(R):
        P, x, y, a, b = _wfr_problem(orc, 6, 7, eta, s=12.0, pid=pid)
        if K is None:
            K, _ = P.dense_kernel()
            acc = np.zeros_like(K)
        sk = P.sparsify()
        rows = np.repeat(np.arange(6), np.diff(sk["row_ptr"]))
        np.add.at(acc, (rows, sk["col_idx"]), sk["val"])
    est = acc / R
    pos = K > 0
    rel = np.abs(est[pos] - K[pos]).sum() / K[pos].sum()
    assert rel < 0.08, rel
    assert np.all(est[~pos] == 0.0)
