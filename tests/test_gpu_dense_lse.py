"""GPU parity of dense Sinkhorn in log-sum-exp form (Alg. 1 / Alg. 2 with
binary32 potentials) against the oracle's FP64 log-domain dense iterations.

FP32: objective within 1e-5 relative.  At eps = 0.1 the log form must agree
with the plain dense GPU iterations.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2306_06581_gb300 import inputs  # noqa: E402


@pytest.fixture(scope="module")
def S():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2306_06581_gb300 import build, sparsink
    build.build()
    return sparsink


def _r32(w):
    f = lambda z: np.asarray(z, np.float32).astype(np.float64)
    return f(w.x), f(w.y), f(w.a), f(w.b)


def _close_iters(g, o):
    return abs(g - o) <= max(3, 0.05 * o)


def test_dense_lse_ot_small_eps(S, orc):
    w = inputs.ot_gmm(1200, d=3, k=8, seed=33, eps=0.01)
    x, y, a, b = _r32(w)
    P = orc.OracleProblem(a, b, 0.01, 1.0, math.inf, x=x, y=y)
    o = orc.dense_sinkhorn(P, tol=1e-5, max_iter=20000, log_domain=True)
    g = S.sinkhorn_dense(a, b, x, y, eps=0.01, tol=1e-5, max_iter=20000, dtype="f32", log_domain=1)
    assert o["info"]["status"] == 0 and g["status"] == 0
    assert _close_iters(g["iters"], o["info"]["iters"]), (g["iters"], o["info"]["iters"])
    assert abs(g["obj"] - o["obj"]) <= 1e-5 * abs(o["obj"])
    al = g["alpha"].cpu().numpy().astype(np.float64)
    d = (al - al.mean()) - (o["alpha"] - o["alpha"].mean())
    assert np.abs(d).max() < 5e-5


def test_dense_lse_uot_small_eps(S, orc):
    w = inputs.uot_n20000(n=1000)
    x, y, a, b = _r32(w)
    P = orc.OracleProblem(a, b, 0.01, 1.0, 1.0, x=x, y=y)
    o = orc.dense_sinkhorn(P, tol=1e-5, max_iter=20000, log_domain=True)
    g = S.sinkhorn_dense(a, b, x, y, eps=0.01, lam=1.0, tol=1e-5, max_iter=20000, dtype="f32", log_domain=1)
    assert o["info"]["status"] == 0 and g["status"] == 0
    assert _close_iters(g["iters"], o["info"]["iters"]), (g["iters"], o["info"]["iters"])
    assert abs(g["obj"] - o["obj"]) <= 1e-5 * abs(o["obj"])
    for k in ("kl_a", "kl_b", "mass", "transport"):
        assert abs(g[k] - o["terms"][k]) <= 1e-4 * abs(o["terms"][k]) + 1e-9, k
    # potentials of UOT are unique (no gauge)
    al = g["alpha"].cpu().numpy().astype(np.float64)
    assert np.abs(al - o["alpha"]).max() < 5e-5


@pytest.mark.parametrize("lam", [math.inf, 1.0])
def test_dense_lse_equals_plain_at_moderate_eps(S, lam):
    w = inputs.small_problem(n=900, m=700, d=4, seed=43, eps=0.1, mass_b=1.0 if math.isinf(lam) else 1.5)
    x, y, a, b = _r32(w)
    kw = dict(eps=0.1, lam=lam, tol=1e-5, max_iter=5000, dtype="f32")
    pl = S.sinkhorn_dense(a, b, x, y, **kw)
    lg = S.sinkhorn_dense(a, b, x, y, log_domain=1, **kw)
    assert abs(pl["iters"] - lg["iters"]) <= max(2, 0.05 * pl["iters"])
    assert abs(pl["obj"] - lg["obj"]) <= 2e-6 * abs(pl["obj"])
    assert torch.allclose(pl["alpha"], lg["alpha"], rtol=0, atol=2e-5)


def test_dense_lse_cost_matrix_equals_points(S):
    w = inputs.small_problem(n=300, m=260, d=3, seed=44, eps=0.01)
    x, y, a, b = _r32(w)
    C = ((x[:, None, :] - y[None, :, :]) ** 2).sum(-1)
    kw = dict(eps=0.01, tol=1e-5, max_iter=20000, dtype="f32", log_domain=1)
    gp = S.sinkhorn_dense(a, b, x, y, **kw)
    gc = S.sinkhorn_dense(a, b, C_=C, **kw)
    assert gp["status"] == 0 and gc["status"] == 0
    assert abs(gp["iters"] - gc["iters"]) <= 2
    assert abs(gp["obj"] - gc["obj"]) <= 1e-5 * abs(gp["obj"])
