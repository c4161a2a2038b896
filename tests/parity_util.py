"""Element-wise comparison of FP32 GPU potentials with the FP64 oracle's.

Both sides run exactly K iterations from u = v = 1 (tolerance 0), so the two
pairs differ by rounding alone, not by where each side decided to stop.  OT
potentials are unique only up to (alpha + c, beta - c), but both sides start
from the same pair and apply the same updates, so no gauge is removed here;
UOT potentials have no gauge at all.

Tolerance (FP32 against FP64, stated once for all callers): one half-iteration
forms q_i = sum_j K~_ij v_j over N_i <= N stored elements in binary32, a
relative error of at most N 2^-24 (about sqrt(N) 2^-24 in practice); u = a / q
and its log add a few ulp more.  The Sinkhorn map contracts earlier errors by
a factor kappa < 1 per iteration (kappa ~ 0.9 at the 100-200 iterations these
problems take to reach 1e-5), so the accumulated relative error of u stays
below N 2^-24 / (1 - kappa), i.e. |alpha_gpu - alpha_fp64| <= eps * 10 N 2^-24
(times phi for UOT, which only lowers it).  Entries whose row or column is
unreachable (-inf) must be -inf on both sides.
"""
import math

import numpy as np


def fp32_potential_bound(eps, max_row_nnz):
    """eps * 10 N 2^-24: the accumulated FP32 error of the potentials (module docstring)."""
    return eps * 10.0 * max(int(max_row_nnz), 1) * 2.0 ** -24


def compare_potentials(g_alpha, g_beta, o_alpha, o_beta, bound):
    """Max |difference| of alpha and of beta; the -inf patterns must agree."""
    ga, gb = np.asarray(g_alpha, np.float64), np.asarray(g_beta, np.float64)
    oa, ob = np.asarray(o_alpha, np.float64), np.asarray(o_beta, np.float64)
    fa, fb = np.isfinite(oa), np.isfinite(ob)
    assert np.array_equal(fa, np.isfinite(ga)) and np.array_equal(fb, np.isfinite(gb))
    da = float(np.abs(ga[fa] - oa[fa]).max()) if fa.any() else 0.0
    db = float(np.abs(gb[fb] - ob[fb]).max()) if fb.any() else 0.0
    assert da <= bound and db <= bound, (da, db, bound)
    return da, db


def max_nnz(sketch):
    """Largest row or column count of an oracle sketch."""
    return int(max(np.diff(sketch["row_ptr"]).max(), np.diff(sketch["col_ptr"]).max()))


def fixed_k(run_gpu, orc, P, sketch, K, log_domain=False):
    """The GPU solve and the oracle solve, each stopped after exactly K iterations."""
    g = run_gpu(tol=0.0, max_iter=K, check_every=K, raise_on_error=False)
    o = orc.spar_sink(P, tol=0.0, max_iter=K, log_domain=log_domain, sketch=sketch)
    assert g["iters"] == o["info"]["iters"] == K, (g["iters"], o["info"]["iters"], K)
    return g, o


__all__ = ["fp32_potential_bound", "compare_potentials", "max_nnz", "fixed_k", "math"]
