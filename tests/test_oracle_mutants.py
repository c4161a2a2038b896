"""The pins catch plausible mistakes: each case plants one mistake in a copy
of the oracle (on the CPU, in a temporary directory), runs the pins that
should notice it, and expects them to fail.  The product code is not
involved."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CASES = [
    # (what, file in oracle/ ["#k": the k-th occurrence of the text, else its only one],
    #  correct text, planted text, pins)
    ("OT factor without the square root of a", "sparsink_oracle.c",
     "for (int32_t i = 0; i < n; ++i) sa[i] = sqrtf((float)P->a[i]);",
     "for (int32_t i = 0; i < n; ++i) sa[i] = (float)P->a[i];", "test_oracle_sampler.py"),
    ("UOT exponent lam / (lam + eps) in the probabilities", "sparsink_oracle.c",
     "S->gamma32 = (float)(P->lambda / t);", "S->gamma32 = (float)(P->lambda / (P->lambda + P->eps));",
     "test_oracle_sampler.py"),
    ("keep rule inflated by 1%", "sparsink_oracle.c", "return u < praw;", "return u <= praw * 1.01f;",
     "test_oracle_sampler.py"),
    ("value K p* instead of K / p*", "sparsink_oracle.c", "if (val) val[c] = Kij / (double)ps;",
     "if (val) val[c] = Kij * (double)ps;", "test_oracle_sampler.py"),
    ("Alg. 2 exponent lam / (2 lam + eps), scaling iterations", "sparsink_oracle.c#1",
     "const double phi = isinf(lambda) ? 1.0 : lambda / (lambda + eps);",
     "const double phi = isinf(lambda) ? 1.0 : lambda / (2.0 * lambda + eps);", "test_oracle_sinkhorn.py"),
    ("Alg. 2 exponent lam / (2 lam + eps), log-domain iterations", "sparsink_oracle.c#2",
     "const double phi = isinf(lambda) ? 1.0 : lambda / (lambda + eps);",
     "const double phi = isinf(lambda) ? 1.0 : lambda / (2.0 * lambda + eps);", "test_oracle_sinkhorn.py"),
    ("entropy without the -1", "sparsink_oracle.c", "ne += T * (lt - 1.0);", "ne += T * lt;",
     "test_oracle_sinkhorn.py"),
    ("transport term <T, sqrt C>", "sparsink_oracle.c", "tr += T * cost[k];", "tr += T * sqrt(cost[k]);",
     "test_oracle_gaussian.py"),
    ("FP64 cost over the first coordinate only", "sparsink_oracle.c",
     "for (int k = 0; k < P->d; ++k) {\n    double t = P->x", "for (int k = 0; k < 1; ++k) {\n    double t = P->x",
     "test_oracle_gaussian.py"),
    ("KL term sign", "sparsink_oracle.c", "return x * log(x / y) - x + y;", "return x * log(x / y) + x - y;",
     "test_oracle_sinkhorn.py"),
    ("skip sampler: gap rate log q instead of log(1 - q)", "sparsink_oracle.c",
     "const float L = full ? 0.0f : orc_log1m32(q);", "const float L = full ? 0.0f : orc_log32(q);",
     "test_oracle_skip.py"),
    ("skip sampler: acceptance p instead of p / q", "sparsink_oracle.c",
     "const float acc = full ? p : p / q;", "const float acc = p;", "test_oracle_skip.py"),
    ("skip sampler: one word for gap and acceptance", "sparsink_oracle.c",
     "const float V = (float)(w[1] >> 8) * 0x1p-24f;", "const float V = (float)(w[0] >> 8) * 0x1p-24f;",
     "test_oracle_skip.py"),
    ("WFR: cos instead of cos^2", "sparsink_oracle.c", "return -2.0 * log(cos(z));", "return -log(cos(z));",
     "test_oracle_wfr.py"),
    ("WFR: decision angle d / eta", "sparsink_oracle.c",
     "S->inv2eta32 = is_wfr(P) ? (float)(1.0 / (2.0 * P->eta)) : 0.0f;",
     "S->inv2eta32 = is_wfr(P) ? (float)(1.0 / P->eta) : 0.0f;", "test_oracle_wfr.py"),
    ("equal probabilities without the budget s", "sparsink_oracle.c",
     "for (int32_t i = 0; i < n; ++i) rowf[i] = S->s32 * S->scale32;",
     "for (int32_t i = 0; i < n; ++i) rowf[i] = S->scale32;", "test_oracle_randsink.py"),
    ("cost divisor: maximum over half of the columns", "sparsink_oracle.c",
     "for (int32_t j = 0; j < m; ++j) {\n      float d32 = raw_cost32(P, i, j);",
     "for (int32_t j = 0; j < m / 2; ++j) {\n      float d32 = raw_cost32(P, i, j);", "test_oracle_sampler.py"),
    ("decision draw: counter words i and j >> 2 swapped", "sparsink_oracle.c",
     "uint32_t ctr[4] = {j >> 2, i, pid, 0x5A17u};", "uint32_t ctr[4] = {i, j >> 2, pid, 0x5A17u};",
     "test_oracle_rng.py"),
    ("decision draw: word 0 of the block for every column", "sparsink_oracle.c",
     "return out[j & 3u] >> 8;", "return out[0] >> 8;", "test_oracle_rng.py"),
    ("UOT decision factor exp(+D kappa)", "sparsink_oracle.c",
     "if (!is_wfr(P)) return orc_exp32(-(dd * S->kappa32));", "if (!is_wfr(P)) return orc_exp32(dd * S->kappa32);",
     "test_oracle_sampler.py"),
    ("UOT normaliser Z without the kernel factor", "sparsink_oracle.c",
     "sa_add(&part, uot_weight(P, rowf, colf, S, i, j));", "sa_add(&part, rowf[i] * colf[j]);",
     "test_oracle_sampler.py"),
    ("sparse-problem value with -eps sum T log p*", "oracle.py",
     'return r1, r1 + eps * terms["logp"]', 'return r1, r1 - eps * terms["logp"]', "test_oracle_sparsink.py"),
    ("UOT objective with the KL term of a only", "oracle.py",
     'r1 += lam * (terms["kl_a"] + terms["kl_b"])', 'r1 += lam * terms["kl_a"]', "test_oracle_sinkhorn.py"),
    ("log-domain UOT update without the exponent phi", "sparsink_oracle.c",
     "alpha[i] = L[i] > -INFINITY ? phi * (eps * log(a[i]) - eps * L[i]) : -INFINITY;",
     "alpha[i] = L[i] > -INFINITY ? (eps * log(a[i]) - eps * L[i]) : -INFINITY;", "test_oracle_sparsink.py"),
    ("sparse cost without the divisor in the value path", "sparsink_oracle.c",
     "return is_wfr(P) ? wfr_cost64(P, d) : d / cost_divisor(P, S);",
     "return is_wfr(P) ? wfr_cost64(P, d) : d;", "test_oracle_sparsink.py"),
    ("Philox: nine rounds", "sparsink_oracle.c", "for (int r = 0; r < 10; ++r) {",
     "for (int r = 0; r < 9; ++r) {", "test_oracle_rng.py"),
    ("exact sum: ties not to even", "sparsink_oracle.c", "if (round_bit && (sticky || (mant & 1u))) {",
     "if (round_bit && sticky) {", "test_oracle_specmath.py"),
    ("exact sum: sticky scan skips a bit", "sparsink_oracle.c", "for (int p = hb - 54; p >= 0 && !sticky; --p)",
     "for (int p = hb - 55; p >= 0 && !sticky; --p)", "test_oracle_specmath.py"),
    ("KL(0 | y) taken as 0", "sparsink_oracle.c", "if (x == 0.0) return y;", "if (x == 0.0) return 0.0;",
     "test_oracle_sinkhorn.py"),
    ("UOT stopping residual without the power 1/phi", "sparsink_oracle.c",
     "double ui = (phi == 1.0) ? u[i] : pow(u[i], 1.0 / phi);", "double ui = u[i];", "test_oracle_sinkhorn.py"),
    ("log-domain UOT stopping residual without 1/phi", "sparsink_oracle.c#1",
     "res += fabs(exp(alpha[i] * ie / phi + L[i]) - a[i]);", "res += fabs(exp(alpha[i] * ie + L[i]) - a[i]);",
     "test_oracle_sinkhorn.py"),
    ("log-domain residual of a capped run without 1/phi", "sparsink_oracle.c#2",
     "res += fabs(exp(alpha[i] * ie / phi + L[i]) - a[i]);", "res += fabs(exp(alpha[i] * ie + L[i]) - a[i]);",
     "test_oracle_sinkhorn.py"),
    ("log-sum-exp without its shift back", "sparsink_oracle.c", "  return mx + log(acc);", "  return log(acc);",
     "test_oracle_sinkhorn.py"),
    ("network: points scaled by 1 / cost_max", "mlp_oracle.py", "s = 1.0 / np.sqrt(cost_max)",
     "s = 1.0 / cost_max", "test_oracle_mlp.py"),
    ("network: mass feature a_i without n", "mlp_oracle.py", "(len(sw) * np.asarray(sw, np.float64))[:, None]",
     "(np.asarray(sw, np.float64))[:, None]", "test_oracle_mlp.py"),
    ("network: loss not weighted by a", "mlp_oracle.py", "a = np.where(fin, np.asarray(sw, np.float64), 0.0)",
     "a = np.where(fin, 1.0, 0.0)", "test_oracle_mlp.py"),
    ("IBP: arithmetic instead of geometric mean", "ibp_oracle.py",
     "logq += w[k] * np.log(np.where(Kv[k] > 0, Kv[k], 1.0))",
     "logq += w[k] * np.where(Kv[k] > 0, Kv[k], 1.0)", "test_oracle_ibp.py"),
    ("IBP: K instead of K^T for v", "ibp_oracle.py",
     "vs[k] = _safe_div(np.asarray(bs[k], np.float64), Ks[k].T @ us[k])",
     "vs[k] = _safe_div(np.asarray(bs[k], np.float64), Ks[k] @ us[k])", "test_oracle_ibp.py"),
]


def _copy(tmp_path):
    for sub in ("oracle", "paper_2306_06581_gb300", "tests"):
        shutil.copytree(os.path.join(ROOT, sub), os.path.join(tmp_path, sub),
                        ignore=shutil.ignore_patterns("*.so", "*.o", "_build", "__pycache__", "*.tmp"))


def _pins(tmp_path, files):
    return subprocess.run([sys.executable, "-m", "pytest", *[os.path.join("tests", f) for f in files], "-q", "-x",
                           "-m", "not gpu", "-p", "no:cacheprovider", "-W", "ignore::RuntimeWarning"],
                          cwd=tmp_path, capture_output=True, text=True, timeout=600)


def test_unchanged_copy_passes(tmp_path):
    # the control: in the copy, with nothing planted, every pin above passes (so a failure below is the mistake's)
    _copy(tmp_path)
    r = _pins(tmp_path, sorted({c[4] for c in CASES}))
    assert r.returncode == 0, (r.stdout[-2000:], r.stderr[-2000:])


@pytest.mark.parametrize("what,fn,good,bad,pins", CASES, ids=[c[0] for c in CASES])
def test_planted_mistake_is_caught(tmp_path, what, fn, good, bad, pins):
    _copy(tmp_path)
    fn, _, k = fn.partition("#")
    path = os.path.join(tmp_path, "oracle", fn)
    src = open(path).read()
    parts = src.split(good)
    # the correct text is where the case expects it: once, or at least k times for "#k"
    assert len(parts) > int(k) if k else len(parts) == 2, what
    k = int(k or 1)
    open(path, "w").write(good.join(parts[:k]) + bad + good.join(parts[k:]))
    r = _pins(tmp_path, [pins])
    assert r.returncode == 1 and " failed" in r.stdout, (what, r.stdout[-2000:], r.stderr[-2000:])
