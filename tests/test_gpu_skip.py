"""GPU parity of the skip sampler (geometric gaps with thinning)
against the oracle's restatement of the same stream:

- pattern (CSR, CSC, csr_pos) bit-exact, values within the element
  sampler's tolerances (FP64 1e-12, FP32 2e-6 relative);
- Spar-Sink on the skip sketch: objective within 1e-9 (FP64) / 1e-5 (FP32)
  relative of the oracle's Alg. 3 on its own skip sketch;
- 200000 points (the 8-component mixture workload): nnz equal to the
  oracle's count and sampled rows bit-exact, in the configuration the
  benchmark runs;
- UOT (Eq. pij-uot): patterns bit-exact and the Alg. 4 objective within
  1e-5 of the oracle's on its own skip sketch.
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


def _round32(w):
    f = lambda z: np.asarray(z, np.float32).astype(np.float64)
    return f(w.x), f(w.y), f(w.a), f(w.b)


def _check_pattern(g, o):
    assert g["nnz"] == o["nnz"]
    assert np.array_equal(g["row_ptr"].cpu().numpy(), o["row_ptr"])
    assert np.array_equal(g["col_idx"].cpu().numpy(), o["col_idx"])
    assert np.array_equal(g["col_ptr"].cpu().numpy(), o["col_ptr"])
    assert np.array_equal(g["row_idx"].cpu().numpy(), o["row_idx"])
    assert np.array_equal(g["csr_pos"].cpu().numpy(), o["perm"])


@pytest.mark.parametrize("n,m,d,sf", [(300, 517, 3, 0.08), (1, 1, 2, 5.0), (257, 129, 10, 0.3),
                                      (640, 700, 3, 0.01), (40, 50, 2, 60.0)])
def test_skip_pattern_bit_exact_f32(S, orc, n, m, d, sf):
    w = inputs.small_problem(n=n, m=m, d=d, seed=n + 2 * m)
    x, y, a, b = _round32(w)
    s = max(3.0, sf * n * m)
    g = S.sparsify_kernel(a, b, x, y, eps=0.1, s=s, dtype="f32", seed=99, problem_id=3, sampler="skip")
    o = orc.OracleProblem(a, b, 0.1, s, math.inf, x=x, y=y, seed=99, pid=3).sparsify(sampler="skip")
    _check_pattern(g, o)
    assert np.allclose(g["val"].cpu().numpy(), o["val"], rtol=2e-6, atol=0)
    assert np.allclose(g["valT"].cpu().numpy(), o["valT"], rtol=2e-6, atol=0)


def test_skip_pattern_f64_values(S, orc):
    w = inputs.ot_n1000()
    g = S.sparsify_kernel(w.a, w.b, w.x, w.y, eps=w.eps, s=w.s, dtype="f64", seed=w.seed, sampler="skip")
    o = orc.OracleProblem(w.a, w.b, w.eps, w.s, math.inf, x=w.x, y=w.y, seed=w.seed).sparsify(sampler="skip")
    _check_pattern(g, o)
    assert np.allclose(g["val"].cpu().numpy(), o["val"], rtol=1e-12, atol=0)


@pytest.mark.parametrize("dtype,rtol", [("f64", 1e-9), ("f32", 1e-5)])
def test_skip_spar_sink_objective(S, orc, dtype, rtol):
    w = inputs.ot_n1000()
    x, y, a, b = _round32(w) if dtype == "f32" else (w.x, w.y, w.a, w.b)
    r = S.spar_sink_ot(a, b, x, y, eps=w.eps, s=w.s, tol=1e-6, dtype=dtype, seed=w.seed, sampler="skip")
    P = orc.OracleProblem(a, b, w.eps, w.s, math.inf, x=x, y=y, seed=w.seed)
    o = orc.spar_sink(P, tol=1e-6, sketch=P.sparsify(sampler="skip"))
    assert r["nnz"] == o["sketch"]["nnz"]
    assert abs(r["obj"] - o["obj"]) <= rtol * abs(o["obj"])
    assert abs(r["iters"] - o["info"]["iters"]) <= max(2, 0.05 * o["info"]["iters"])


def test_skip_log_domain_matches_oracle(S, orc):
    w = inputs.ot_gmm(20000, 3, 8, 3, 0.01, 16.0, 1e-5, "f32")
    x, y, a, b = _round32(w)
    r = S.spar_sink_ot(a, b, x, y, eps=w.eps, s=w.s, tol=1e-5, dtype="f32", log_domain=1, seed=w.seed,
                       max_iter=5000, sampler="skip")
    P = orc.OracleProblem(a, b, w.eps, w.s, math.inf, x=x, y=y, seed=w.seed)
    o = orc.spar_sink(P, tol=1e-5, max_iter=5000, log_domain=True, sketch=P.sparsify(sampler="skip"))
    assert r["nnz"] == o["sketch"]["nnz"]
    assert abs(r["obj"] - o["obj"]) <= 1e-5 * abs(o["obj"])


def test_skip_200k_rows_and_count(S, orc):
    w = inputs.ot_n200000(dtype="f32")
    x, y, a, b = _round32(w)
    g = S.sparsify_kernel(a, b, x, y, eps=w.eps, s=w.s, dtype="f32", seed=w.seed, sampler="skip")
    P = orc.OracleProblem(a, b, w.eps, w.s, math.inf, x=x, y=y, seed=w.seed)
    cnt, nnz = P.skip_count()
    assert g["nnz"] == nnz
    rp = g["row_ptr"].cpu().numpy()
    assert np.array_equal(np.diff(rp), cnt)
    ci = g["col_idx"].cpu().numpy()
    val = g["val"].cpu().numpy()
    for i in np.random.default_rng(0).choice(w.n, 40, replace=False):
        r = P.skip_row(int(i))
        assert np.array_equal(ci[rp[i]:rp[i + 1]], r["cols"]), i
        # binary32 value path at eps = 0.01: |C / eps| up to 100 amplifies the
        # rounding of C (the element sampler's large-size test uses the same bound)
        assert np.allclose(val[rp[i]:rp[i + 1]], r["val"], rtol=2e-5, atol=1e-37)


@pytest.mark.parametrize("n,m,d,lam", [(300, 517, 3, 1.0), (257, 129, 10, 0.5), (7, 5, 2, 2.0)])
def test_skip_uot_pattern_bit_exact(S, orc, n, m, d, lam):
    w = inputs.small_problem(n=n, m=m, d=d, seed=n + m, mass_b=1.5)
    x, y, a, b = _round32(w)
    s = max(10.0, 0.08 * n * m)
    g = S.sparsify_kernel(a, b, x, y, eps=0.1, s=s, lam=lam, dtype="f32", seed=5, problem_id=2, sampler="skip")
    o = orc.OracleProblem(a, b, 0.1, s, lam, x=x, y=y, seed=5, pid=2).sparsify(sampler="skip")
    _check_pattern(g, o)
    assert np.allclose(g["val"].cpu().numpy(), o["val"], rtol=2e-6, atol=0)


def test_skip_uot_solve_matches_oracle(S, orc):
    w = inputs.uot_n20000(n=3000)
    x, y, a, b = _round32(w)
    r = S.spar_sink_uot(a, b, x, y, eps=w.eps, lam=w.lam, s=w.s, tol=1e-5, dtype="f32", seed=w.seed,
                        sampler="skip")
    P = orc.OracleProblem(a, b, w.eps, w.s, w.lam, x=x, y=y, seed=w.seed)
    o = orc.spar_sink(P, tol=1e-5, sketch=P.sparsify(sampler="skip"))
    assert r["nnz"] == o["sketch"]["nnz"]
    assert abs(r["obj"] - o["obj"]) <= 1e-5 * abs(o["obj"])
    # potentials element by element after the oracle's iteration count on both sides (UOT: no gauge)
    K = o["info"]["iters"]
    run = lambda **e: S.spar_sink_uot(a, b, x, y, eps=w.eps, lam=w.lam, s=w.s, dtype="f32", seed=w.seed,
                                      sampler="skip", **e)
    gk, ok = fixed_k(run, orc, P, o["sketch"], K)
    da, db = compare_potentials(gk["alpha"].cpu(), gk["beta"].cpu(), ok["alpha"], ok["beta"],
                                fp32_potential_bound(w.eps, max_nnz(o["sketch"])))
    print(f"UOT n=3000 skip FP32 potentials after {K} iterations: max |d alpha| {da:.2e}, |d beta| {db:.2e}")
