"""Pins for the oracle's scaling iterations (Alg. 1, Alg. 2), the log-domain
form and the objective terms.

Each check compares with something computed another way:
- entropic OT is sandwiched by the linear-programming optimum
  (scipy.optimize.linprog, or brute force over permutations):
  OT - eps(1 + 2 log n) <= OT_eps <= OT - eps, since H(T) in [1, 1 + 2 log n];
- strong duality: OT_eps equals the maximum of the concave dual
  g(alpha, beta) = a.alpha + b.beta - eps sum exp((alpha_i+beta_j-C_ij)/eps),
  found by a generic quasi-Newton optimiser; the paper's f = g + eps
  (Eq. dual-ot) so f* = OT_eps + eps;
- UOT: the 1x1 problem has the closed form log t = (lam log a + lam log b - C)/(2lam+eps);
  the primal equals the dual lam a.(1-e^{-alpha/lam}) + lam b.(1-e^{-beta/lam})
  - eps sum e^{(alpha+beta-C)/eps}; a direct numerical minimisation of the primal
  of Eq. (ruot) agrees; lam -> infinity recovers OT (sec. 2.2);
- eps -> infinity gives T -> a b^T (sec. 2.1);
- the log-domain iteration reproduces the plain one;
- KL and H against scipy.special.kl_div / entr.
"""
import itertools
import math

import numpy as np
import pytest
from scipy import optimize, special

from paper_2306_06581_gb300 import inputs


def _sqdist(x, y):
    return ((x[:, None, :] - y[None, :, :]) ** 2).sum(-1)


def _dense(orc, a, b, C, eps, lam=math.inf, tol=1e-12, max_iter=100000):
    P = orc.OracleProblem(a, b, eps, 1.0, lam, C_=C, cost_norm=0)
    return orc.dense_sinkhorn(P, tol=tol, max_iter=max_iter)


def _lp_value(a, b, C):
    n, m = C.shape
    A_eq = np.zeros((n + m, n * m))
    for i in range(n):
        A_eq[i, i * m:(i + 1) * m] = 1
    for j in range(m):
        A_eq[n + j, j::m] = 1
    r = optimize.linprog(C.ravel(), A_eq=A_eq, b_eq=np.concatenate([a, b]), bounds=(0, None),
                         method="highs")
    assert r.status == 0
    return r.fun


def test_lp_brute_force_and_sandwich(orc):
    rng = np.random.default_rng(0)
    n = 6
    x, y = rng.normal(size=(n, 2)), rng.normal(size=(n, 2))
    C = _sqdist(x, y)
    C = C / C.max()
    a = b = np.full(n, 1.0 / n)
    ot = min(sum(C[i, p[i]] for i in range(n)) for p in itertools.permutations(range(n))) / n
    assert abs(ot - _lp_value(a, b, C)) < 1e-9
    for eps in [0.3, 0.1, 0.03, 0.01]:
        r = _dense(orc, a, b, C, eps)
        assert r["info"]["status"] == 0
        assert ot - eps * (1 + 2 * math.log(n)) - 1e-9 <= r["obj"] <= ot - eps + 1e-9
    # eps -> 0: <T, C> -> OT
    r = _dense(orc, a, b, C, 0.005)
    assert abs(r["terms"]["transport"] - ot) < 0.02 * ot


def test_lp_sandwich_nonuniform(orc):
    rng = np.random.default_rng(1)
    n, m = 7, 5
    C = rng.uniform(0, 1, (n, m))
    a = rng.uniform(0.1, 1, n); a /= a.sum()
    b = rng.uniform(0.1, 1, m); b /= b.sum()
    ot = _lp_value(a, b, C)
    for eps in [0.1, 0.02]:
        r = _dense(orc, a, b, C, eps)
        assert ot - eps * (1 + 2 * math.log(max(n, m))) - 1e-9 <= r["obj"] <= ot - eps + 1e-9


def _dual_g(al_be, a, b, C, eps):
    n = a.size
    al, be = al_be[:n], al_be[n:]
    Z = np.exp((al[:, None] + be[None, :] - C) / eps)
    val = a @ al + b @ be - eps * Z.sum()
    grad = np.concatenate([a - Z.sum(1), b - Z.sum(0)])
    return -val, -grad


def test_strong_duality_against_generic_optimiser(orc):
    rng = np.random.default_rng(2)
    n, m = 8, 6
    C = rng.uniform(0, 1, (n, m))
    a = rng.uniform(0.2, 1, n); a /= a.sum()
    b = rng.uniform(0.2, 1, m); b /= b.sum()
    eps = 0.1
    r = _dense(orc, a, b, C, eps)
    opt = optimize.minimize(_dual_g, np.zeros(n + m), args=(a, b, C, eps), jac=True,
                            method="L-BFGS-B", options={"gtol": 1e-13, "ftol": 1e-15, "maxiter": 20000})
    assert abs(-opt.fun - r["obj"]) < 1e-9
    # the oracle's own potentials are dual-optimal; the paper's f = g + eps (Eq. dual-ot)
    g_star = -_dual_g(np.concatenate([r["alpha"], r["beta"]]), a, b, C, eps)[0]
    assert abs(g_star - r["obj"]) < 1e-10
    f_star = g_star + eps
    assert abs(f_star - (a @ r["alpha"] + b @ r["beta"])) < 1e-10
    # marginals of the plan
    T = np.exp((r["alpha"][:, None] + r["beta"][None, :] - C) / eps)
    assert np.abs(T.sum(1) - a).sum() <= 1e-12 and np.abs(T.sum(0) - b).sum() < 1e-12


def test_eps_to_infinity_gives_product_plan(orc):
    rng = np.random.default_rng(3)
    C = rng.uniform(0, 1, (5, 4))
    a = np.array([0.1, 0.2, 0.3, 0.25, 0.15]); b = np.array([0.4, 0.3, 0.2, 0.1])
    r = _dense(orc, a, b, C, 1e5)
    T = r["u"][:, None] * r["K"] * r["v"][None, :]
    assert np.abs(T - np.outer(a, b)).max() < 1e-5


def test_uot_one_by_one_closed_form(orc):
    for a_, b_, c_, lam, eps in [(0.7, 1.9, 0.3, 1.0, 0.05), (2.0, 0.5, 1.2, 0.1, 0.1), (1.0, 1.0, 0.0, 5, 0.01)]:
        r = _dense(orc, np.array([a_]), np.array([b_]), np.array([[c_]]), eps, lam)
        t = math.exp((lam * math.log(a_) + lam * math.log(b_) - c_) / (2 * lam + eps))
        T = r["u"][0] * r["K"][0, 0] * r["v"][0]
        assert abs(T / t - 1) < 1e-10


def _uot_primal(T, a, b, C, eps, lam):
    T = T.reshape(C.shape)
    return ((T * C).sum() + lam * special.kl_div(T.sum(1), a).sum() + lam * special.kl_div(T.sum(0), b).sum()
            - eps * (special.entr(T).sum() + T.sum()))


def test_uot_primal_dual_and_direct_minimisation(orc):
    rng = np.random.default_rng(4)
    n, m = 4, 3
    C = rng.uniform(0, 1, (n, m))
    a = rng.uniform(0.2, 1, n); b = 1.5 * rng.dirichlet(np.ones(m))
    for lam, eps in [(1.0, 0.05), (0.3, 0.2)]:
        r = _dense(orc, a, b, C, eps, lam)
        al, be = r["alpha"], r["beta"]
        dual = (lam * a @ (1 - np.exp(-al / lam)) + lam * b @ (1 - np.exp(-be / lam))
                - eps * np.exp((al[:, None] + be[None, :] - C) / eps).sum())
        assert abs(dual - r["obj"]) < 1e-9
        T0 = np.outer(a, b) / a.sum()
        opt = optimize.minimize(_uot_primal, T0.ravel(), args=(a, b, C, eps, lam), method="L-BFGS-B",
                                bounds=[(1e-300, None)] * (n * m),
                                options={"ftol": 1e-15, "gtol": 1e-12, "maxiter": 50000})
        assert abs(opt.fun - r["obj"]) < 1e-7
        # first-order conditions (appendix): u^{(lam+eps)/lam} (K v) = a
        phi = lam / (lam + eps)
        assert np.allclose(r["u"] ** (1 / phi) * (r["K"] @ r["v"]), a, rtol=1e-9)


def test_uot_tends_to_ot(orc):
    rng = np.random.default_rng(5)
    C = rng.uniform(0, 1, (6, 6))
    a = rng.dirichlet(np.ones(6)); b = rng.dirichlet(np.ones(6))
    ot = _dense(orc, a, b, C, 0.1)
    uot = _dense(orc, a, b, C, 0.1, lam=1e6, tol=1e-13)
    assert abs(uot["obj"] - ot["obj"]) < 1e-4
    assert np.allclose(uot["alpha"] - uot["alpha"].mean(), ot["alpha"] - ot["alpha"].mean(), atol=1e-4)


def test_objective_terms_against_scipy(orc):
    rng = np.random.default_rng(6)
    n, m = 5, 4
    T = rng.uniform(0, 0.1, (n, m)); T[1, 2] = 0.0
    T[3, :] = 0.0                      # a row with no mass: KL(0 | a_3) = a_3
    C = rng.uniform(0, 1, (n, m))
    a = rng.uniform(0.05, 0.5, n); b = rng.uniform(0.05, 0.5, m)
    ps = rng.uniform(0.1, 1, (n, m)).astype(np.float32)
    row_ptr = np.arange(n + 1) * m
    col_idx = np.tile(np.arange(m), n)
    with np.errstate(divide="ignore"):
        logT = np.log(T).ravel()
    t = orc.objective_terms(row_ptr, col_idx, logT, C.ravel(), ps.ravel(), a, b)
    assert abs(t["transport"] - (T * C).sum()) < 1e-15
    assert abs(t["neg_entropy"] - (-(special.entr(T).sum() + T.sum()))) < 1e-14
    assert abs(t["kl_a"] - special.kl_div(T.sum(1), a).sum()) < 1e-14
    assert abs(t["kl_a"] - (special.kl_div(np.delete(T.sum(1), 3), np.delete(a, 3)).sum() + a[3])) < 1e-14
    assert abs(t["kl_b"] - special.kl_div(T.sum(0), b).sum()) < 1e-14
    assert abs(t["logp"] - (T * np.log(ps.astype(np.float64))).sum()) < 1e-14


@pytest.mark.parametrize("lam", [math.inf, 1.0])
def test_log_domain_equals_plain(orc, lam):
    w = inputs.small_problem(n=120, m=100, d=4, seed=7, eps=0.1, mass_b=1.0 if math.isinf(lam) else 1.5)
    P = orc.OracleProblem(w.a, w.b, 0.1, w.s, lam, x=w.x, y=w.y)
    sk = P.sparsify()
    pl = orc.spar_sink(P, tol=1e-11, max_iter=20000, sketch=sk)
    lg = orc.spar_sink(P, tol=1e-11, max_iter=20000, sketch=sk, log_domain=True)
    assert pl["info"]["iters"] == lg["info"]["iters"]
    fin = np.isfinite(pl["alpha"])
    assert np.array_equal(fin, np.isfinite(lg["alpha"]))
    assert np.abs(pl["alpha"][fin] - lg["alpha"][fin]).max() < 1e-12
    assert abs(pl["obj"] - lg["obj"]) < 1e-12


def test_fixed_point_independent_of_start(orc):
    rng = np.random.default_rng(8)
    C = rng.uniform(0, 1, (9, 7))
    a = rng.dirichlet(np.ones(9)); b = rng.dirichlet(np.ones(7))
    K = np.exp(-C / 0.1)
    u1, v1, _ = orc.sinkhorn_dense(K, a, b, 0.1, tol=1e-13, max_iter=100000)
    u2, v2, _ = orc.sinkhorn_dense(K, a, b, 0.1, tol=1e-13, max_iter=100000,
                                   u0=rng.uniform(0.5, 2, 9), v0=rng.uniform(0.5, 2, 7))
    T1 = u1[:, None] * K * v1[None]
    T2 = u2[:, None] * K * v2[None]
    assert np.abs(T1 - T2).max() < 1e-12


def test_stopping_rules(orc):
    rng = np.random.default_rng(9)
    C = rng.uniform(0, 1, (20, 15))
    a = rng.dirichlet(np.ones(20)); b = rng.dirichlet(np.ones(15))
    K = np.exp(-C / 0.05)
    u, v, info = orc.sinkhorn_dense(K, a, b, 0.05, tol=1e-8, max_iter=100000)
    assert info["status"] == 0 and info["residual"] <= 1e-8
    T = u[:, None] * K * v[None]
    assert abs(np.abs(T.sum(1) - a).sum() - info["residual"]) < 1e-15
    assert np.abs(T.sum(0) - b).sum() < 1e-14
    # the previous pair did not satisfy the tolerance (first pair that does is returned)
    u2, v2, info2 = orc.sinkhorn_dense(K, a, b, 0.05, tol=1e-8, max_iter=info["iters"] - 1)
    assert info2["status"] == 1 and info2["residual"] > 1e-8
    # paper's rule (Alg. 1): ||du||_1 + ||dv||_1 <= delta
    u3, v3, info3 = orc.sinkhorn_dense(K, a, b, 0.05, tol=1e-6, max_iter=100000, stop_rule=orc.STOP_DELTA_UV)
    assert info3["status"] == 0 and info3["residual"] <= 1e-6


def test_empty_row_is_unreachable_not_nan(orc):
    # An empty row of K~ (no sampled element) carries mass that no plan on the
    # sketch can move: u_i = 0 (alpha_i = -inf), the row is left out of the
    # stopping residual and its mass is reported.  Balanced OT stays solvable
    # when that mass is negligible; UOT always has a fixed point.
    w = inputs.small_problem(n=50, m=50, d=3, seed=10)
    a = w.a.copy()
    a[7] = 1e-30                      # sqrt(a_7) tiny: row 7 never sampled
    a /= a.sum()
    bu = np.full(50, 1.0 / 50)
    P = orc.OracleProblem(a, bu, 0.1, 1500.0, math.inf, x=w.x, y=w.y)
    r = orc.spar_sink(P, tol=1e-8, max_iter=5000)
    sk = r["sketch"]
    assert sk["row_ptr"][8] == sk["row_ptr"][7]
    assert (np.diff(sk["col_ptr"]) > 0).all()
    assert r["info"]["status"] == 0
    assert r["alpha"][7] == -np.inf and np.isfinite(r["obj"])
    assert r["info"]["unreach_a"] == a[7]
    # UOT with empty rows and columns of non-negligible mass
    b = w.b.copy()
    b[3] = 1e-30
    P = orc.OracleProblem(a, 1.5 * b / b.sum(), 0.1, 300.0, 1.0, x=w.x, y=w.y)
    r = orc.spar_sink(P, tol=1e-9, max_iter=20000)
    sk = r["sketch"]
    empty_c = np.diff(sk["col_ptr"]) == 0
    assert empty_c[3] and r["info"]["status"] == 0
    assert np.isneginf(r["beta"][empty_c]).all() and np.isfinite(r["obj"])
    assert abs(r["info"]["unreach_b"] - P.b[empty_c].sum()) < 1e-15


@pytest.mark.parametrize("lam", [math.inf, 1.0])
def test_dense_log_domain_equals_plain(orc, lam):
    w = inputs.small_problem(n=60, m=50, d=3, seed=17, eps=0.1, mass_b=1.0 if math.isinf(lam) else 1.5)
    P = orc.OracleProblem(w.a, w.b, 0.1, 1.0, lam, x=w.x, y=w.y)
    pl = orc.dense_sinkhorn(P, tol=1e-11, max_iter=20000)
    lg = orc.dense_sinkhorn(P, tol=1e-11, max_iter=20000, log_domain=True)
    assert pl["info"]["iters"] == lg["info"]["iters"]
    assert np.abs(pl["alpha"] - lg["alpha"]).max() < 1e-12
    assert abs(pl["obj"] - lg["obj"]) < 1e-12


def test_dense_log_domain_small_eps_lp_sandwich(orc):
    # eps = 1e-3 on a cost normalised to [0, 1]: exp(-C/eps) underflows binary64
    # for C > 0.745, so only the log form is usable.  Uniform weights, n = 7:
    # OT is the best permutation (Birkhoff), and OT - eps(1 + 2 log n) <= OT_eps <= OT - eps.
    rng = np.random.default_rng(21)
    n = 7
    # a permuted, slightly moved copy of x: one best matching with a clear margin
    x = rng.uniform(0, 1, (n, 2)); y = x[rng.permutation(n)] + 0.02 * rng.standard_normal((n, 2))
    a = np.full(n, 1.0 / n); b = np.full(n, 1.0 / n)
    C = ((x[:, None] - y[None]) ** 2).sum(-1)
    C = C / C.max()
    assert (np.exp(-C / 1e-3) == 0).any()
    ot = min(sum(C[i, p[i]] for i in range(n)) / n for p in itertools.permutations(range(n)))
    eps = 1e-3
    P = orc.OracleProblem(a, b, eps, 1.0, math.inf, C_=C, cost_norm=0)
    r = orc.dense_sinkhorn(P, tol=1e-12, max_iter=500000, log_domain=True)
    assert r["info"]["status"] == 0
    assert ot - eps * (1 + 2 * math.log(n)) - 1e-9 <= r["obj"] <= ot - eps + 1e-9
    assert abs(r["terms"]["transport"] - ot) < 5e-3
    T = np.exp((r["alpha"][:, None] + r["beta"][None]) / eps - C / eps)
    assert np.abs(T.sum(1) - a).sum() < 1e-11 and np.abs(T.sum(0) - b).sum() < 1e-11


def _sketch_rows(sk):
    return np.repeat(np.arange(sk["n"]), np.diff(sk["row_ptr"]))


@pytest.mark.parametrize("lam", [1.0, 0.3])
def test_uot_stopping_residual(orc, lam):
    # Reading c-1: UOT marginals are penalised, not constrained, so the stopping
    # residual is the fixed-point one of Alg. 2: u = (a / Kv)^phi holds exactly
    # when u^{1/phi} (Kv) = a, with phi = lam / (lam + eps).  It is checked here
    # from the returned pair, recomputed with numpy, not with the oracle's code.
    rng = np.random.default_rng(11)
    eps = 0.1
    phi = lam / (lam + eps)
    C = rng.uniform(0, 1, (18, 13))
    a = rng.dirichlet(np.ones(18)); b = 1.5 * rng.dirichlet(np.ones(13))
    K = np.exp(-C / eps)
    u, v, info = orc.sinkhorn_dense(K, a, b, eps, lam=lam, tol=1e-9, max_iter=100000)
    assert info["status"] == 0
    res = np.abs(u ** (1 / phi) * (K @ v) - a).sum()
    assert res <= 1e-9 and abs(res - info["residual"]) <= 1e-15
    # the column side holds right after the v-update of the same iteration
    assert np.abs(v ** (1 / phi) * (K.T @ u) - b).sum() < 1e-13
    # the plain-OT residual of the same pair is far from zero: the marginals are not matched
    assert np.abs(u * (K @ v) - a).sum() > 1e-3
    # the first pair under tol is returned: the one before it is not
    _, _, info2 = orc.sinkhorn_dense(K, a, b, eps, lam=lam, tol=1e-9, max_iter=info["iters"] - 1)
    assert info2["status"] == 1 and info2["residual"] > 1e-9

    # log-domain form on a sketch: the residual of (alpha, beta) with u = e^{alpha/eps}
    w = inputs.small_problem(n=40, m=30, d=3, seed=12)
    P = orc.OracleProblem(w.a, 1.5 * w.b, eps, 400.0, lam, x=w.x, y=w.y, seed=5)
    sk = P.sparsify()
    rows = _sketch_rows(sk)

    def log_residual(al, be):
        q = np.zeros(sk["n"])
        np.add.at(q, rows, np.exp(sk["logval"] + be[sk["col_idx"]] / eps))
        ok = q > 0
        return np.abs(np.exp(al[ok] / (eps * phi)) * q[ok] - P.a[ok]).sum()

    al, be, li = orc.sinkhorn_log_sparse(sk, P.a, P.b, eps, lam=lam, tol=1e-9, max_iter=100000)
    assert li["status"] == 0
    r = log_residual(al, be)
    assert r <= 1e-9 and abs(r - li["residual"]) <= 1e-12
    # a capped, unconverged run reports the same residual of its returned pair
    al3, be3, li3 = orc.sinkhorn_log_sparse(sk, P.a, P.b, eps, lam=lam, tol=1e-9, max_iter=3)
    assert li3["status"] == 1
    r3 = log_residual(al3, be3)
    assert r3 > 1e-6 and abs(r3 - li3["residual"]) <= 1e-12 * r3
