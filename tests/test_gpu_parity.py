"""GPU parity: the CUDA path through the C ABI against the FP64 CPU oracle.

- sampling pattern (CSR and CSC indices, csr_pos): bit-exact;
- sketch values: FP64 within 1e-12 relative, FP32 within 2e-6 relative;
- Spar-Sink / dense Sinkhorn, FP64: iterations within 1, potentials within
  1e-9, objective terms within 1e-10 relative;
- FP32: objective within 1e-5 relative (the tolerance the method is held to
  in FP32), iterations within max(3, 3%); potentials element by element after
  the same fixed number of iterations on both sides, within the FP32 bound of
  tests/parity_util.py (eps 10 N 2^-24, N the largest row or column count).
Sizes span several row/column tiles with ragged tails.
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
    """Inputs as binary32 values (both sides then see identical numbers)."""
    f = lambda z: None if z is None else np.asarray(z, np.float32).astype(np.float64)
    return f(w.x), f(w.y), f(w.a), f(w.b)


def _oracle_problem(orc, x, y, a, b, eps, lam, s, seed=0x5EED, pid=0, C_=None, cost_norm=1):
    return orc.OracleProblem(a, b, eps, s, lam, x=x, y=y, C_=C_, cost_norm=cost_norm, seed=seed, pid=pid)


def _check_pattern(g, o):
    assert g["nnz"] == o["nnz"]
    assert np.array_equal(g["row_ptr"].cpu().numpy(), o["row_ptr"])
    assert np.array_equal(g["col_idx"].cpu().numpy(), o["col_idx"])
    assert np.array_equal(g["col_ptr"].cpu().numpy(), o["col_ptr"])
    assert np.array_equal(g["row_idx"].cpu().numpy(), o["row_idx"])
    assert np.array_equal(g["csr_pos"].cpu().numpy(), o["perm"])


@pytest.mark.parametrize("n,m,d,lam", [(300, 517, 3, math.inf), (300, 517, 3, 1.0), (1, 1, 2, math.inf),
                                       (5, 3, 4, 0.5), (257, 129, 10, math.inf), (131, 260, 5, 2.0)])
def test_pattern_bit_exact_f32(S, orc, n, m, d, lam):
    w = inputs.small_problem(n=n, m=m, d=d, seed=n + m, mass_b=1.0 if math.isinf(lam) else 1.5)
    x, y, a, b = _round32(w)
    s = max(10.0, 0.08 * n * m)
    g = S.sparsify_kernel(a, b, x, y, eps=0.1, s=s, lam=lam, dtype="f32", seed=123, problem_id=7)
    o = _oracle_problem(orc, x, y, a, b, 0.1, lam, s, seed=123, pid=7).sparsify()
    _check_pattern(g, o)
    assert np.allclose(g["val"].cpu().numpy(), o["val"], rtol=2e-6, atol=0)
    assert np.allclose(g["valT"].cpu().numpy(), o["valT"], rtol=2e-6, atol=0)


@pytest.mark.parametrize("lam", [math.inf, 1.0])
def test_pattern_bit_exact_f64_values(S, orc, lam):
    w = inputs.ot_n1000()
    s = w.s
    g = S.sparsify_kernel(w.a, w.b, w.x, w.y, eps=w.eps, s=s, lam=lam, dtype="f64", seed=w.seed)
    o = _oracle_problem(orc, w.x, w.y, w.a, w.b, w.eps, lam, s, seed=w.seed).sparsify()
    _check_pattern(g, o)
    assert np.allclose(g["val"].cpu().numpy(), o["val"], rtol=1e-12, atol=0)


def test_pattern_dense_cost_input(S, orc):
    w = inputs.small_problem(n=90, m=70, d=3, seed=5)
    x, y, a, b = _round32(w)
    Cm = ((x[:, None, :] - y[None]) ** 2).sum(-1)
    for lam in (math.inf, 1.0):
        g = S.sparsify_kernel(a, b, C_=Cm, eps=0.1, s=800.0, lam=lam, dtype="f64")
        o = _oracle_problem(orc, None, None, a, b, 0.1, lam, 800.0, C_=Cm).sparsify()
        _check_pattern(g, o)
        assert np.allclose(g["val"].cpu().numpy(), o["val"], rtol=1e-12)


def test_spar_sink_ot_f64_matches_oracle(S, orc):
    w = inputs.ot_n1000()
    g = S.spar_sink_ot(w.a, w.b, w.x, w.y, eps=w.eps, s=w.s, tol=w.tol, max_iter=5000, dtype="f64", seed=w.seed)
    P = _oracle_problem(orc, w.x, w.y, w.a, w.b, w.eps, math.inf, w.s, seed=w.seed)
    o = orc.spar_sink(P, tol=w.tol, max_iter=5000)
    assert g["status"] == 0 and o["info"]["status"] == 0
    assert abs(g["iters"] - o["info"]["iters"]) <= 1
    assert g["nnz"] == o["sketch"]["nnz"]
    if g["iters"] == o["info"]["iters"]:
        al = g["alpha"].cpu().numpy()
        fin = np.isfinite(o["alpha"])
        assert np.array_equal(fin, np.isfinite(al))
        assert np.abs(al[fin] - o["alpha"][fin]).max() < 1e-9
        for k in ("transport", "neg_entropy", "logp", "mass"):
            assert abs(g[k] - o["terms"][k]) <= 1e-10 * max(1.0, abs(o["terms"][k])), k
    assert abs(g["obj"] - o["obj"]) <= 1e-8 * abs(o["obj"])
    assert abs(g["obj_sparse"] - o["obj_sparse"]) <= 1e-8 * abs(o["obj_sparse"])
    assert g["residual"] <= w.tol


def test_spar_sink_uot_f32_matches_oracle(S, orc):
    w = inputs.uot_n20000(n=1500)
    x, y, a, b = _round32(w)
    g = S.spar_sink_uot(a, b, x, y, eps=w.eps, lam=w.lam, s=w.s, tol=w.tol, max_iter=5000, dtype="f32")
    P = _oracle_problem(orc, x, y, a, b, w.eps, w.lam, w.s)
    o = orc.spar_sink(P, tol=w.tol, max_iter=5000)
    assert g["status"] == 0 and o["info"]["status"] == 0
    assert g["nnz"] == o["sketch"]["nnz"]
    assert abs(g["iters"] - o["info"]["iters"]) <= max(3, 0.03 * o["info"]["iters"])
    assert abs(g["obj"] - o["obj"]) <= 1e-5 * abs(o["obj"])
    assert abs(g["obj_sparse"] - o["obj_sparse"]) <= 1e-5 * abs(o["obj_sparse"])
    for k in ("kl_a", "kl_b", "mass", "transport"):
        assert abs(g[k] - o["terms"][k]) <= 1e-4 * abs(o["terms"][k]) + 1e-9, k
    # potentials element by element after the oracle's iteration count on both sides (UOT: no gauge)
    K = o["info"]["iters"]
    run = lambda **e: S.spar_sink_uot(a, b, x, y, eps=w.eps, lam=w.lam, s=w.s, dtype="f32", **e)
    gk, ok = fixed_k(run, orc, P, o["sketch"], K)
    da, db = compare_potentials(gk["alpha"].cpu(), gk["beta"].cpu(), ok["alpha"], ok["beta"],
                                fp32_potential_bound(w.eps, max_nnz(o["sketch"])))
    print(f"UOT n=1500 FP32 potentials after {K} iterations: max |d alpha| {da:.2e}, |d beta| {db:.2e}")


def test_spar_sink_ot_f32_matches_oracle(S, orc):
    w = inputs.ot_gmm(3000, d=3, k=8, seed=11, eps=0.05, s_factor=16.0)
    x, y, a, b = _round32(w)
    g = S.spar_sink_ot(a, b, x, y, eps=w.eps, s=w.s, tol=1e-5, max_iter=20000, dtype="f32")
    o = orc.spar_sink(_oracle_problem(orc, x, y, a, b, w.eps, math.inf, w.s), tol=1e-5, max_iter=20000)
    assert g["nnz"] == o["sketch"]["nnz"]
    assert g["status"] == o["info"]["status"] == 0
    assert abs(g["iters"] - o["info"]["iters"]) <= max(3, 0.03 * o["info"]["iters"])
    assert abs(g["obj"] - o["obj"]) <= 1e-5 * abs(o["obj"])
    # potentials element by element after the oracle's iteration count on both sides
    K = o["info"]["iters"]
    P = _oracle_problem(orc, x, y, a, b, w.eps, math.inf, w.s)
    run = lambda **e: S.spar_sink_ot(a, b, x, y, eps=w.eps, s=w.s, dtype="f32", **e)
    gk, ok = fixed_k(run, orc, P, o["sketch"], K)
    da, db = compare_potentials(gk["alpha"].cpu(), gk["beta"].cpu(), ok["alpha"], ok["beta"],
                                fp32_potential_bound(w.eps, max_nnz(o["sketch"])))
    print(f"OT n=3000 FP32 potentials after {K} iterations: max |d alpha| {da:.2e}, |d beta| {db:.2e}")


@pytest.mark.parametrize("lam,dtype", [(math.inf, "f64"), (1.0, "f64"), (math.inf, "f32"), (1.0, "f32")])
def test_dense_sinkhorn_matches_oracle(S, orc, lam, dtype):
    w = inputs.small_problem(n=700, m=333, d=5, seed=3, eps=0.1, mass_b=1.0 if math.isinf(lam) else 1.5)
    x, y, a, b = _round32(w) if dtype == "f32" else (w.x, w.y, w.a, w.b)
    g = S.sinkhorn_dense(a, b, x, y, eps=0.1, lam=lam, tol=1e-6 if dtype == "f64" else 1e-5, max_iter=5000, dtype=dtype)
    P = _oracle_problem(orc, x, y, a, b, 0.1, lam, 1.0)
    o = orc.dense_sinkhorn(P, tol=1e-6 if dtype == "f64" else 1e-5, max_iter=5000)
    assert g["status"] == 0
    if dtype == "f64":
        assert abs(g["iters"] - o["info"]["iters"]) <= 1
        assert abs(g["obj"] - o["obj"]) <= 1e-9 * abs(o["obj"])
        if g["iters"] == o["info"]["iters"]:
            assert np.abs(g["alpha"].cpu().numpy() - o["alpha"]).max() < 1e-9
    else:
        assert abs(g["iters"] - o["info"]["iters"]) <= max(3, 0.03 * o["info"]["iters"])
        assert abs(g["obj"] - o["obj"]) <= 1e-5 * abs(o["obj"])


def test_all_kept_equals_dense(S):
    w = inputs.small_problem(n=200, m=150, d=3, seed=9, eps=0.2)
    sp = S.spar_sink_ot(w.a, w.b, w.x, w.y, eps=0.2, s=1e12, tol=1e-9, max_iter=5000, dtype="f64")
    de = S.sinkhorn_dense(w.a, w.b, w.x, w.y, eps=0.2, tol=1e-9, max_iter=5000, dtype="f64")
    assert sp["nnz"] == 200 * 150
    assert sp["iters"] == de["iters"]
    assert abs(sp["obj"] - de["obj"]) < 1e-11
    assert torch.allclose(sp["alpha"], de["alpha"], rtol=0, atol=1e-10)


def test_deterministic(S):
    w = inputs.uot_n20000(n=2000)
    r1 = S.spar_sink_uot(w.a, w.b, w.x, w.y, eps=w.eps, lam=w.lam, s=w.s, tol=w.tol, dtype="f32")
    r2 = S.spar_sink_uot(w.a, w.b, w.x, w.y, eps=w.eps, lam=w.lam, s=w.s, tol=w.tol, dtype="f32")
    assert r1["iters"] == r2["iters"] and r1["obj"] == r2["obj"] and r1["residual"] == r2["residual"]
    assert torch.equal(r1["alpha"], r2["alpha"])


def test_not_converged_and_numeric(S):
    w = inputs.small_problem(n=300, m=300, d=3, seed=4, eps=0.05)
    r = S.spar_sink_ot(w.a, w.b, w.x, w.y, eps=0.05, s=w.s, tol=1e-14, max_iter=3, dtype="f32")
    assert r["status"] == S.SPS_NOT_CONVERGED and r["iters"] == 3 and math.isfinite(r["obj"])
    a = w.a.copy()
    a[5] = np.nan
    with pytest.raises(S.SpsError, match="NUMERIC"):
        S.spar_sink_ot(a, w.b, w.x, w.y, eps=0.05, s=w.s, dtype="f32")


def test_empty_rows_reported(S, orc):
    w = inputs.small_problem(n=400, m=400, d=3, seed=8)
    a = w.a.copy()
    a[:3] = 1e-30
    a /= a.sum()
    b = np.full(400, 1 / 400)
    g = S.spar_sink_ot(a, b, w.x, w.y, eps=0.1, s=20000.0, tol=1e-8, max_iter=5000, dtype="f64")
    o = orc.spar_sink(_oracle_problem(orc, w.x, w.y, a, b, 0.1, math.inf, 20000.0), tol=1e-8, max_iter=5000)
    al = g["alpha"].cpu().numpy()
    assert np.isneginf(al[:3]).all() and np.isneginf(o["alpha"][:3]).all()
    assert abs(g["unreach_a"] - o["info"]["unreach_a"]) < 1e-18
    assert abs(g["obj"] - o["obj"]) <= 1e-9 * abs(o["obj"])


def test_full_size_uot_rows_bit_exact(S, orc):
    """The n = m = 20000 UOT workload: the GPU pattern of sampled rows against
    the oracle row by row (the oracle's exact Z is the full n*m sum)."""
    w = inputs.uot_n20000()
    x, y, a, b = _round32(w)
    g = S.sparsify_kernel(a, b, x, y, eps=w.eps, s=w.s, lam=w.lam, dtype="f32", seed=w.seed)
    P = _oracle_problem(orc, x, y, a, b, w.eps, w.lam, w.s, seed=w.seed)
    rp = g["row_ptr"].cpu().numpy()
    ci = g["col_idx"].cpu().numpy()
    vals = g["val"].float().cpu().numpy()
    rng = np.random.default_rng(0)
    rows = np.concatenate([[0, 1, w.n - 1], rng.choice(w.n, 40, replace=False)])
    for i in rows:
        r = P.sample_row(int(i))
        assert np.array_equal(ci[rp[i]:rp[i + 1]], r["cols"]), i
        assert np.allclose(vals[rp[i]:rp[i + 1]], r["val"], rtol=2e-6)
    # nnz is consistent with E nnz = sum p* <= s
    assert abs(g["nnz"] - w.s) < 6 * math.sqrt(w.s)


@pytest.mark.parametrize("lam,n,m,kd", [(math.inf, 3000, 2500, "f32"), (1.0, 3000, 2800, "f32"),
                                          (math.inf, 20000, 20000, "bf16"), (1.0, 900, 700, "f64")])
def test_single_pass_sketch_equals_two_pass(S, lam, n, m, kd):
    """The single-pass sketch (padded slots, then compaction) gives the
    two-pass sketch bit for bit: CSR, CSC, values and the CSR positions."""
    w = inputs.small_problem(n=n, m=m, d=3, seed=91, eps=0.1, mass_b=1.0 if math.isinf(lam) else 1.5)
    x, y, a, b = _round32(w)
    kw = dict(eps=0.1, s=w.s, lam=lam, dtype="f64" if kd == "f64" else "f32", kdtype=kd, seed=17)
    one = S.sparsify_kernel(a, b, x, y, sketch_mode=0, **kw)
    two = S.sparsify_kernel(a, b, x, y, sketch_mode=1, **kw)
    assert one["nnz"] == two["nnz"]
    for k in ("row_ptr", "col_idx", "col_ptr", "row_idx", "csr_pos"):
        assert torch.equal(one[k], two[k]), k
    assert torch.equal(one["val"].view(torch.uint8), two["val"].view(torch.uint8))
    assert torch.equal(one["valT"].view(torch.uint8), two["valT"].view(torch.uint8))


@pytest.mark.parametrize("lam", [math.inf, 1.0])
def test_single_pass_log_domain_solve_equals_two_pass(S, lam):
    w = inputs.small_problem(n=2500, m=2200, d=3, seed=92, eps=0.01, mass_b=1.0 if math.isinf(lam) else 1.5)
    x, y, a, b = _round32(w)
    f = S.spar_sink_ot if math.isinf(lam) else (lambda *z, **k: S.spar_sink_uot(*z, lam=lam, **k))
    kw = dict(eps=0.01, s=w.s, tol=1e-5, max_iter=5000, dtype="f32", seed=3, log_domain=1)
    r1 = f(a, b, x, y, sketch_mode=0, **kw)
    r2 = f(a, b, x, y, sketch_mode=1, **kw)
    assert r1["nnz"] == r2["nnz"] and r1["iters"] == r2["iters"] and r1["obj"] == r2["obj"]
    assert torch.equal(r1["alpha"], r2["alpha"])


@pytest.mark.parametrize("n,m,d,lam", [(300, 257, 5, 1.0), (513, 700, 10, 0.5), (64, 2000, 2, 2.0), (400, 350, 3, math.inf)])
def test_exact_normalisers_bit_equal(S, orc, n, m, d, lam):
    """The sampling normalisers are exact sums rounded once: UOT Z of Eq. (pij-uot)
    (a fixed-point window per thread plus a full-range slow path on the GPU, the
    oracle's own exact sum on the CPU), OT sum sqrt(a) and sum sqrt(b)."""
    w = inputs.small_problem(n=n, m=m, d=d, seed=3 * n + m, mass_b=1.0 if math.isinf(lam) else 1.5)
    x, y, a, b = _round32(w)
    s = max(10.0, 0.05 * n * m)
    g = S.sparsify_kernel(a, b, x, y, eps=0.1, s=s, lam=lam, dtype="f32", seed=5, problem_id=1)
    P = _oracle_problem(orc, x, y, a, b, 0.1, lam, s, seed=5, pid=1)
    _, _, sc = P.factors()
    assert g["sum1"] == sc.sum1 and g["sum1"] > 0.0
    if math.isinf(lam):
        assert g["sum2"] == sc.sum2 and g["sum2"] > 0.0


@pytest.mark.parametrize("sampler,sketch_mode", [("element", 0), ("element", 1), ("skip", 0)])
def test_sparsify_values_ignore_log_domain_params(S, sampler, sketch_mode):
    """sparsify_kernel returns K~ itself whatever the params' log_domain says (the
    stabilised solve keeps only log K~ internally, the sparsifier never does)."""
    w = inputs.small_problem(n=400, m=300, d=3, seed=17)
    x, y, a, b = _round32(w)
    kw = dict(eps=0.1, s=0.1 * 400 * 300, dtype="f32", seed=3, sampler=sampler, sketch_mode=sketch_mode)
    g0 = S.sparsify_kernel(a, b, x, y, **kw)
    g1 = S.sparsify_kernel(a, b, x, y, log_domain=1, **kw)
    assert g0["nnz"] == g1["nnz"] > 0
    for k in ("col_idx", "row_idx", "csr_pos"):
        assert torch.equal(g0[k], g1[k]), k
    assert torch.equal(g0["val"].view(torch.int32), g1["val"].view(torch.int32))
    assert torch.equal(g0["valT"].view(torch.int32), g1["valT"].view(torch.int32))
