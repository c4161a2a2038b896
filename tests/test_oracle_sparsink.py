"""Statistical pins for Spar-Sink as a whole (Alg. 3 / Alg. 4).

- Theorem 1 / 2 bound the error of the estimate by c eps sqrt(n^{3-2 alpha}/s):
  the relative error against dense Sinkhorn falls as s grows, at least as
  fast as s^{-1/2} (checked with slack on the mean over seeds);
- Theorem 3: Spar-Sink needs the same order of iterations as Sinkhorn;
- the sparse problem's own value (cost C~ = C + eps log p*) and the literal
  output line of Alg. 3 both converge to OT_eps.
"""
import math

import numpy as np
import pytest


def _setup(n=200, d=5, seed=0):
    rng = np.random.default_rng(seed)
    x = rng.uniform(0, 1, (n, d))
    y = rng.uniform(0, 1, (n, d))
    a = rng.uniform(0.2, 1, n); a /= a.sum()
    b = rng.uniform(0.2, 1, n); b /= b.sum()
    return x, y, a, b


@pytest.mark.parametrize("lam", [math.inf, 1.0])
def test_error_falls_with_budget(orc, lam):
    n, eps = 200, 0.1
    x, y, a, b = _setup(n)
    if not math.isinf(lam):
        b = 1.5 * b
    P = orc.OracleProblem(a, b, eps, 1.0, lam, x=x, y=y)
    dense = orc.dense_sinkhorn(P, tol=1e-10, max_iter=100000)
    ref = dense["obj"]
    budgets = [16 * n, 32 * n, 64 * n]
    err1, err2, iters = [], [], []
    for s in budgets:
        e1, e2, it = [], [], []
        for r in range(12):
            Ps = orc.OracleProblem(a, b, eps, s, lam, x=x, y=y, seed=100 + r)
            sp = orc.spar_sink(Ps, tol=1e-10, max_iter=100000)
            assert sp["info"]["status"] == 0
            e1.append(abs(sp["obj"] - ref) / abs(ref))
            e2.append(abs(sp["obj_sparse"] - ref) / abs(ref))
            it.append(sp["info"]["iters"])
        err1.append(np.mean(e1)); err2.append(np.mean(e2)); iters.append(np.mean(it))
    for err in (err1, err2):
        assert err[0] > err[1] > err[2]
        assert err[2] / err[0] <= 1.3 * math.sqrt(budgets[0] / budgets[2])
    # the sparse problem's value is the closer estimate at every budget
    assert all(e2 < e1 for e1, e2 in zip(err1, err2))
    # Theorem 3: same order of iterations
    ratio = np.array(iters) / dense["info"]["iters"]
    assert (ratio > 0.5).all() and (ratio < 3.0).all()


def test_uot_spar_sink_close_to_dense(orc):
    n = 150
    x, y, a, b = _setup(n, seed=1)
    P = orc.OracleProblem(a, 1.5 * b, 0.05, 60 * n, 1.0, x=x, y=y, seed=9)
    sp = orc.spar_sink(P, tol=1e-10, max_iter=100000)
    de = orc.dense_sinkhorn(P, tol=1e-10, max_iter=100000)
    assert abs(sp["obj_sparse"] - de["obj"]) / abs(de["obj"]) < 0.05


def test_sparse_problem_value_is_the_dual_optimum_on_the_support(orc):
    # Reading c-3: obj_sparse (R2) is the entropic OT value of the sparse problem whose cost is
    # C~ = C + eps log p* on the sampled support S and +inf elsewhere, since K~ = K / p* = exp(-C~/eps).
    # Its concave dual max a.alpha + b.beta - eps sum_{(i,j) in S} exp((alpha_i + beta_j - C~_ij)/eps),
    # maximised here by a generic quasi-Newton method, must equal R2; R1 differs by eps sum T log p*.
    from scipy import optimize
    n = 30
    x, y, a, b = _setup(n, seed=4)
    P = orc.OracleProblem(a, b, 0.1, 12 * n, math.inf, x=x, y=y, seed=3)
    sp = orc.spar_sink(P, tol=1e-12, max_iter=100000)
    sk = sp["sketch"]
    assert sp["info"]["status"] == 0 and sp["info"]["unreach_a"] == 0.0 and np.isfinite(sp["beta"]).all()
    rows = np.repeat(np.arange(n), np.diff(sk["row_ptr"]))
    cols = sk["col_idx"]
    Ct = sk["cost"] + 0.1 * np.log(sk["pstar"].astype(np.float64))
    eps = 0.1

    def neg_dual(z):
        al, be = z[:n], z[n:]
        E = np.exp((al[rows] + be[cols] - Ct) / eps)
        g = a @ al + b @ be - eps * E.sum()
        ga = a - np.bincount(rows, E, n)
        gb = b - np.bincount(cols, E, n)
        return -g, -np.concatenate([ga, gb])

    opt = optimize.minimize(neg_dual, np.zeros(2 * n), jac=True, method="L-BFGS-B",
                            options={"gtol": 1e-13, "ftol": 1e-16, "maxiter": 50000})
    assert abs(-opt.fun - sp["obj_sparse"]) < 1e-8 * abs(sp["obj_sparse"])
    assert abs(sp["obj_sparse"] - sp["obj"] - eps * sp["terms"]["logp"]) < 1e-12
    assert abs(sp["terms"]["logp"]) > 1e-3          # the two readings differ on this sketch


def test_sparse_uot_value_is_the_dual_optimum_on_the_support(orc):
    # Readings c-3 and c-6 for Alg. 4: R2 of a UOT sketch equals the maximum of
    # lam a.(1 - e^{-alpha/lam}) + lam b.(1 - e^{-beta/lam}) - eps sum_S exp((alpha_i + beta_j - C~_ij)/eps)
    # over the sampled support S, with C~ = C + eps log p* (generic quasi-Newton maximiser).
    from scipy import optimize
    n, eps, lam = 30, 0.1, 0.7
    x, y, a, b = _setup(n, seed=5)
    b = 1.5 * b
    P = orc.OracleProblem(a, b, eps, 12 * n, lam, x=x, y=y, seed=8)
    sp = orc.spar_sink(P, tol=1e-12, max_iter=100000)
    sk = sp["sketch"]
    assert sp["info"]["status"] == 0 and np.isfinite(sp["alpha"]).all() and np.isfinite(sp["beta"]).all()
    rows = np.repeat(np.arange(n), np.diff(sk["row_ptr"]))
    cols = sk["col_idx"]
    Ct = sk["cost"] + eps * np.log(sk["pstar"].astype(np.float64))

    def neg_dual(z):
        al, be = z[:n], z[n:]
        E = np.exp((al[rows] + be[cols] - Ct) / eps)
        ea, eb = np.exp(-al / lam), np.exp(-be / lam)
        g = lam * a @ (1 - ea) + lam * b @ (1 - eb) - eps * E.sum()
        ga = a * ea - np.bincount(rows, E, n)
        gb = b * eb - np.bincount(cols, E, n)
        return -g, -np.concatenate([ga, gb])

    opt = optimize.minimize(neg_dual, np.zeros(2 * n), jac=True, method="L-BFGS-B",
                            options={"gtol": 1e-13, "ftol": 1e-16, "maxiter": 50000})
    assert abs(-opt.fun - sp["obj_sparse"]) < 1e-8 * abs(sp["obj_sparse"])
    # the oracle's own potentials attain it
    assert abs(-neg_dual(np.concatenate([sp["alpha"], sp["beta"]]))[0] - sp["obj_sparse"]) < 1e-9


@pytest.mark.parametrize("lam", [math.inf, 0.7])
def test_log_domain_sparse_value_is_the_dual_optimum(orc, lam):
    # The same identity for the log-domain form at eps = 0.01 (where exp(-C/eps) spans ~43 orders of
    # magnitude): R2 equals the maximum of the sparse problem's dual, found by L-BFGS from zero.
    from scipy import optimize
    n, eps = 40, 0.01
    x, y, a, b = _setup(n, seed=6)
    if not math.isinf(lam):
        b = 1.5 * b
    P = orc.OracleProblem(a, b, eps, 12 * n, lam, x=x, y=y, seed=9)
    sp = orc.spar_sink(P, tol=1e-12, max_iter=200000, log_domain=True)
    sk = sp["sketch"]
    assert sp["info"]["status"] == 0 and np.isfinite(sp["alpha"]).all() and np.isfinite(sp["beta"]).all()
    rows = np.repeat(np.arange(n), np.diff(sk["row_ptr"]))
    cols = sk["col_idx"]
    Ct = sk["cost"] + eps * np.log(sk["pstar"].astype(np.float64))

    def neg_dual(z):
        al, be = z[:n], z[n:]
        E = np.exp((al[rows] + be[cols] - Ct) / eps)
        if math.isinf(lam):
            g = a @ al + b @ be - eps * E.sum()
            ga, gb = a - np.bincount(rows, E, n), b - np.bincount(cols, E, n)
        else:
            ea, eb = np.exp(-al / lam), np.exp(-be / lam)
            g = lam * a @ (1 - ea) + lam * b @ (1 - eb) - eps * E.sum()
            ga, gb = a * ea - np.bincount(rows, E, n), b * eb - np.bincount(cols, E, n)
        return -g, -np.concatenate([ga, gb])

    opt = optimize.minimize(neg_dual, np.zeros(2 * n), jac=True, method="L-BFGS-B",
                            options={"gtol": 1e-13, "ftol": 1e-16, "maxiter": 50000})
    assert abs(-opt.fun - sp["obj_sparse"]) < 1e-9 * abs(sp["obj_sparse"])


def test_wfr_uot_value_is_the_dual_optimum_with_unreachable_mass(orc):
    # WFR cost (section 2.2) with eta = 0.25: transport is blocked beyond pi eta, a row and a column of the
    # sketch are empty (reading c-4: their mass is unreachable).  Their KL terms lam a_i are the
    # supremum of lam a_i (1 - e^{-alpha_i/lam}) as alpha_i grows, so R2 still equals the dual optimum.
    from scipy import optimize
    n, eps, lam = 30, 0.1, 0.7
    x, y, a, b = _setup(n, seed=7)
    b = 1.5 * b
    P = orc.OracleProblem(a, b, eps, 12 * n, lam, x=x, y=y, seed=4, cost_kind="wfr", eta=0.25, cost_norm=0)
    sp = orc.spar_sink(P, tol=1e-12, max_iter=100000)
    sk = sp["sketch"]
    assert sp["info"]["status"] == 0
    assert sp["info"]["unreach_a"] > 0 and sp["info"]["unreach_b"] > 0
    assert np.isfinite(sk["cost"]).all()
    rows = np.repeat(np.arange(n), np.diff(sk["row_ptr"]))
    cols = sk["col_idx"]
    Ct = sk["cost"] + eps * np.log(sk["pstar"].astype(np.float64))

    def neg_dual(z):
        al, be = z[:n], z[n:]
        E = np.exp((al[rows] + be[cols] - Ct) / eps)
        ea, eb = np.exp(-al / lam), np.exp(-be / lam)
        g = lam * a @ (1 - ea) + lam * b @ (1 - eb) - eps * E.sum()
        ga, gb = a * ea - np.bincount(rows, E, n), b * eb - np.bincount(cols, E, n)
        return -g, -np.concatenate([ga, gb])

    opt = optimize.minimize(neg_dual, np.zeros(2 * n), jac=True, method="L-BFGS-B",
                            options={"gtol": 1e-13, "ftol": 1e-16, "maxiter": 50000})
    assert abs(-opt.fun - sp["obj_sparse"]) < 1e-9 * abs(sp["obj_sparse"])
