"""GPU parity of the Wasserstein-Fisher-Rao cost (section 2.2) and of the
equal-probability control (Rand-Sink, section 5) against the FP64 oracle.

- WFR, UOT (Eq. pij-uot with the cos power as the decision factor): sampling
  pattern bit-exact for both samplers and several shapes, values within 1e-12
  (FP64) / 2e-6 (FP32) relative; no element is kept where d_ij >= pi eta.
- WFR solves, plain (FP64: iterations within 1, objective within 1e-9; FP32:
  objective within 1e-5 and potentials after a fixed iteration count within
  the FP32 bound of parity_util) and stabilised (eps = 0.01); a source point
  whose every pair is blocked gives an empty row, its mass reported as
  unreachable (reading c-4) on both sides.
- WFR with balanced OT: the separable decision keeps elements whose K is 0;
  their value is 0 (log value -inf) on both sides.
- Equal probabilities (p_ij = 1/(n m)), OT and UOT: pattern bit-exact for both
  samplers, every kept element with the same p*, values within 2e-6 relative
  (or 1e-37 absolute, where K leaves the binary32 normal range), solves as
  above.
The problems are those of the section 5 simulations: masses 5 and 3,
eps = lambda = 0.1, eta set so that about half of the pairs can transport.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2306_06581_gb300 import inputs  # noqa: E402
from parity_util import compare_potentials, fixed_k, fp32_potential_bound, max_nnz  # noqa: E402


@pytest.fixture(scope="module")
def S():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2306_06581_gb300 import build, sparsink
    build.build()
    return sparsink


def _wfr_problem(n, m, d, seed, isolated=False):
    """Section 5 shape: masses 5 and 3; eta = median distance / pi, so that about
    half of the pairs lie within pi eta.  isolated: the first source point is moved
    beyond pi eta of every target (its row of K is empty)."""
    w = inputs.small_problem(n=n, m=m, d=d, seed=seed, mass_a=5.0, mass_b=3.0)
    f = lambda z: np.asarray(z, np.float32).astype(np.float64)
    x, y, a, b = f(w.x), f(w.y), f(w.a), f(w.b)
    dist = np.sqrt(((x[:, None, :] - y[None, :, :]) ** 2).sum(-1))
    eta = float(np.median(dist)) / math.pi
    if isolated:
        x = x.copy()
        x[0] = f(np.full(d, 50.0))
    return x, y, a, b, eta


def _check_pattern(g, o):
    assert g["nnz"] == o["nnz"]
    assert np.array_equal(g["row_ptr"].cpu().numpy(), o["row_ptr"])
    assert np.array_equal(g["col_idx"].cpu().numpy(), o["col_idx"])
    assert np.array_equal(g["col_ptr"].cpu().numpy(), o["col_ptr"])
    assert np.array_equal(g["row_idx"].cpu().numpy(), o["row_idx"])
    assert np.array_equal(g["csr_pos"].cpu().numpy(), o["perm"])


def _wfr_kw(eta):
    return dict(cost_norm=0, cost_kind="wfr", eta=eta)


@pytest.mark.parametrize("sampler", ["element", "skip"])
@pytest.mark.parametrize("n,m,d,dtype", [(300, 257, 5, "f64"), (300, 257, 5, "f32"), (64, 100, 2, "f32"),
                                         (5, 3, 2, "f64")])
def test_wfr_uot_pattern_bit_exact(S, orc, sampler, n, m, d, dtype):
    x, y, a, b, eta = _wfr_problem(n, m, d, seed=n + m)
    s = max(10.0, 0.1 * n * m)
    g = S.sparsify_kernel(a, b, x, y, eps=0.1, s=s, lam=0.1, dtype=dtype, seed=9, problem_id=3, sampler=sampler,
                          cost_norm=S.COST_RAW, cost_kind="wfr", eta=eta)
    P = orc.OracleProblem(a, b, 0.1, s, 0.1, x=x, y=y, seed=9, pid=3, **_wfr_kw(eta))
    o = P.sparsify(sampler=sampler)
    _check_pattern(g, o)
    assert np.all(np.isfinite(o["cost"]))              # nothing kept where d >= pi eta
    rtol = 1e-12 if dtype == "f64" else 2e-6
    assert np.allclose(g["val"].cpu().numpy(), o["val"], rtol=rtol, atol=0)


def test_wfr_ot_keeps_blocked_elements_with_zero_value(S, orc):
    x, y, a, b, eta = _wfr_problem(200, 150, 3, seed=4)
    a, b = a / a.sum(), b / b.sum()
    s = 0.2 * 200 * 150
    g = S.sparsify_kernel(a, b, x, y, eps=0.1, s=s, lam=math.inf, dtype="f64", cost_norm=S.COST_RAW,
                          cost_kind="wfr", eta=eta)
    o = orc.OracleProblem(a, b, 0.1, s, math.inf, x=x, y=y, **_wfr_kw(eta)).sparsify()
    _check_pattern(g, o)
    val = g["val"].cpu().numpy()
    blocked = ~np.isfinite(o["cost"])
    assert blocked.any() and np.all(val[blocked] == 0.0)
    assert np.allclose(val[~blocked], o["val"][~blocked], rtol=1e-12, atol=0)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_wfr_uot_solve_with_an_unreachable_row(S, orc, dtype):
    x, y, a, b, eta = _wfr_problem(400, 350, 5, seed=12, isolated=True)
    s = inputs.s_budget(400, 8.0)
    tol = 1e-6 if dtype == "f64" else 1e-5
    run = lambda **e: S.spar_sink_uot(a, b, x, y, eps=0.1, lam=0.1, s=s, dtype=dtype, cost_norm=S.COST_RAW,
                                      cost_kind="wfr", eta=eta, **e)
    g = run(tol=tol, max_iter=20000)
    P = orc.OracleProblem(a, b, 0.1, s, 0.1, x=x, y=y, **_wfr_kw(eta))
    o = orc.spar_sink(P, tol=tol, max_iter=20000)
    assert g["status"] == 0 and o["info"]["status"] == 0
    assert g["nnz"] == o["sketch"]["nnz"]
    assert np.diff(o["sketch"]["row_ptr"])[0] == 0          # the isolated point's row is empty
    assert g["unreach_a"] == pytest.approx(o["info"]["unreach_a"], rel=1e-6) and g["unreach_a"] >= a[0]
    if dtype == "f64":
        assert abs(g["iters"] - o["info"]["iters"]) <= 1
        assert abs(g["obj"] - o["obj"]) <= 1e-9 * abs(o["obj"])
        for k in ("transport", "neg_entropy", "logp", "kl_a", "kl_b"):
            assert abs(g[k] - o["terms"][k]) <= 1e-9 * max(1.0, abs(o["terms"][k])), k
    else:
        assert abs(g["obj"] - o["obj"]) <= 1e-5 * abs(o["obj"])
        K = o["info"]["iters"]
        gk, ok = fixed_k(run, orc, P, o["sketch"], K)
        da, db = compare_potentials(gk["alpha"].cpu(), gk["beta"].cpu(), ok["alpha"], ok["beta"],
                                    fp32_potential_bound(0.1, max_nnz(o["sketch"])))
        print(f"WFR UOT FP32 potentials after {K} iterations: |d alpha| {da:.2e}, |d beta| {db:.2e}")


def test_wfr_uot_stabilised_solve_matches_oracle(S, orc):
    x, y, a, b, eta = _wfr_problem(500, 450, 3, seed=21)
    s = inputs.s_budget(500, 16.0)
    g = S.spar_sink_uot(a, b, x, y, eps=0.01, lam=0.1, s=s, tol=1e-5, max_iter=20000, dtype="f32", log_domain=1,
                        cost_norm=S.COST_RAW, cost_kind="wfr", eta=eta)
    P = orc.OracleProblem(a, b, 0.01, s, 0.1, x=x, y=y, **_wfr_kw(eta))
    o = orc.spar_sink(P, tol=1e-5, max_iter=20000, log_domain=True)
    assert g["status"] == 0 and o["info"]["status"] == 0
    assert g["nnz"] == o["sketch"]["nnz"]
    assert abs(g["iters"] - o["info"]["iters"]) <= max(3, 0.03 * o["info"]["iters"])
    assert abs(g["obj"] - o["obj"]) <= 1e-5 * abs(o["obj"])


@pytest.mark.parametrize("sampler", ["element", "skip"])
@pytest.mark.parametrize("lam,kind", [(math.inf, "sqeuclid"), (1.0, "sqeuclid"), (0.1, "wfr")])
def test_equal_probabilities_pattern_bit_exact(S, orc, sampler, lam, kind):
    if kind == "wfr":
        x, y, a, b, eta = _wfr_problem(300, 210, 4, seed=5)
        extra_g = dict(cost_norm=S.COST_RAW, cost_kind="wfr", eta=eta)
        extra_o = _wfr_kw(eta)
    else:
        w = inputs.small_problem(n=300, m=210, d=4, seed=5, mass_b=1.0 if math.isinf(lam) else 1.5)
        f = lambda z: np.asarray(z, np.float32).astype(np.float64)
        x, y, a, b = f(w.x), f(w.y), f(w.a), f(w.b)
        extra_g, extra_o = {}, {}
    s = 0.05 * 300 * 210
    g = S.sparsify_kernel(a, b, x, y, eps=0.1, s=s, lam=lam, dtype="f32", sampler=sampler, probs="equal", **extra_g)
    o = orc.OracleProblem(a, b, 0.1, s, lam, x=x, y=y, probs="uniform", **extra_o).sparsify(sampler=sampler)
    _check_pattern(g, o)
    ps = o["pstar"].astype(np.float64)
    assert np.all(ps == ps[0])
    # equal probabilities also keep elements next to the WFR edge, where K = exp(-C/eps) falls below the
    # binary32 normal range (1.2e-38) and the FP32 value flushes to zero: an absolute floor of 1e-37
    assert np.allclose(g["val"].cpu().numpy(), o["val"], rtol=2e-6, atol=1e-37)


@pytest.mark.parametrize("lam", [math.inf, 1.0])
def test_equal_probabilities_solve_matches_oracle(S, orc, lam):
    w = inputs.small_problem(n=600, m=500, d=3, seed=8, mass_b=1.0 if math.isinf(lam) else 1.5)
    f = lambda z: np.asarray(z, np.float32).astype(np.float64)
    x, y, a, b = f(w.x), f(w.y), f(w.a), f(w.b)
    s = 0.1 * 600 * 500
    kw = dict(eps=0.1, s=s, dtype="f32", probs="equal", sampler="skip")
    if math.isinf(lam):
        run = lambda **e: S.spar_sink_ot(a, b, x, y, **kw, **e)
    else:
        run = lambda **e: S.spar_sink_uot(a, b, x, y, lam=lam, **kw, **e)
    g = run(tol=1e-5, max_iter=20000)
    P = orc.OracleProblem(a, b, 0.1, s, lam, x=x, y=y, probs="uniform")
    sk = P.sparsify(sampler="skip")
    o = orc.spar_sink(P, tol=1e-5, max_iter=20000, sketch=sk)
    assert g["status"] == 0 and o["info"]["status"] == 0
    assert g["nnz"] == sk["nnz"]
    assert abs(g["obj"] - o["obj"]) <= 1e-5 * abs(o["obj"])
    assert abs(g["obj_sparse"] - o["obj_sparse"]) <= 1e-5 * abs(o["obj_sparse"])
    K = o["info"]["iters"]
    gk, ok = fixed_k(run, orc, P, sk, K)
    compare_potentials(gk["alpha"].cpu(), gk["beta"].cpu(), ok["alpha"], ok["beta"],
                       fp32_potential_bound(0.1, max_nnz(sk)))
