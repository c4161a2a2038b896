"""GPU: the cost divisor max_ij D_ij found without the full sweep (above 1e8
pairs: grid-bucketed box bounds for d <= 4, radial bounds for larger d)
equals the full sweep's exact maximum.  Checked through the UOT
sampling pattern, which depends on the divisor bit for bit (kappa =
1 / (D_max (2 lam + eps))), and through the OT values, against the oracle's
full n x m maximum.
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


def _r32(z):
    return np.asarray(z, np.float32).astype(np.float64)


def _check_uot(S, orc, x, y, a, b, s):
    g = S.sparsify_kernel(a, b, x, y, eps=0.05, s=s, lam=1.0, dtype="f32", seed=7)
    o = orc.OracleProblem(a, b, 0.05, s, 1.0, x=x, y=y, seed=7).sparsify()
    assert g["nnz"] == o["nnz"]
    assert np.array_equal(g["row_ptr"].cpu().numpy(), o["row_ptr"])
    assert np.array_equal(g["col_idx"].cpu().numpy(), o["col_idx"])
    # binary32 values at eps = 0.05 (|C / eps| up to 20 scales the rounding of C)
    assert np.allclose(g["val"].cpu().numpy(), o["val"], rtol=1e-5, atol=0)


def test_heavy_tailed_uot_pattern(S, orc):
    # 1.21e8 pairs, t-distributed y (nu = 3) in the first 4 coordinates of the 20000-point family
    w = inputs.uot_n20000(n=11000)
    x, y, a, b = _r32(w.x[:, :4]), _r32(w.y[:, :4]), _r32(w.a), _r32(w.b)
    _check_uot(S, orc, x, y, a, b, 16.0 * 11000 * math.log(11000))


def test_heavy_tailed_uot_pattern_d10(S, orc):
    # the 20000-point family itself (d = 10) at 11000 points: the radial bounds
    w = inputs.uot_n20000(n=11000)
    x, y, a, b = _r32(w.x), _r32(w.y), _r32(w.a), _r32(w.b)
    _check_uot(S, orc, x, y, a, b, 16.0 * 11000 * math.log(11000))


def test_gaussian_d6_uot_pattern(S, orc):
    # light tails in d = 6: many points near the largest radius (the radial sets stay large)
    rng = np.random.default_rng(8)
    n = 10500
    x = rng.standard_normal((n, 6))
    y = rng.standard_normal((n, 6)) + 0.3
    a = rng.uniform(0, 1, n)
    b = rng.uniform(0, 1, n)
    _check_uot(S, orc, _r32(x), _r32(y), _r32(a / a.sum()), _r32(b / b.sum() * 1.5), 8.0 * n * math.log(n))


def test_sphere_uot_pattern(S, orc):
    # points on a sphere: a great many pairs within rounding of the maximum
    rng = np.random.default_rng(5)
    n = 11000
    x = rng.standard_normal((n, 3))
    x /= np.linalg.norm(x, axis=1, keepdims=True)
    y = rng.standard_normal((n, 3))
    y /= np.linalg.norm(y, axis=1, keepdims=True)
    a = rng.uniform(0, 1, n)
    b = rng.uniform(0, 1.5, n)
    _check_uot(S, orc, _r32(x), _r32(y), _r32(a / a.sum()), _r32(b / b.sum() * 1.5), 8.0 * n * math.log(n))


def test_mixture_ot_values(S, orc):
    w = inputs.ot_gmm(12000, 3, 16, 9, 0.1, 8.0, 1e-5, "f32")
    x, y, a, b = _r32(w.x), _r32(w.y), _r32(w.a), _r32(w.b)
    g = S.sparsify_kernel(a, b, x, y, eps=0.1, s=w.s, dtype="f32", seed=3)
    o = orc.OracleProblem(a, b, 0.1, w.s, math.inf, x=x, y=y, seed=3).sparsify()
    assert g["nnz"] == o["nnz"]
    assert np.array_equal(g["col_idx"].cpu().numpy(), o["col_idx"])
    assert np.allclose(g["val"].cpu().numpy(), o["val"], rtol=2e-6, atol=0)
