"""The seeded synthetic workloads have the shapes, budgets and value
distributions their recipes state (sizes, dimensions, masses, eps, lambda,
s = factor n ln n, supports of the frame sequence), and they are
reproducible from their seeds.  CPU only; no method arithmetic is involved."""
import math

import numpy as np
import pytest

from paper_2306_06581_gb300 import inputs


def _check_weights(w, mass_a, mass_b):
    assert (w.a > 0).all() and (w.b > 0).all()
    assert math.isclose(w.a.sum(), mass_a, rel_tol=1e-12)
    assert math.isclose(w.b.sum(), mass_b, rel_tol=1e-12)
    # U(0,1) weights before scaling: the ratio of mean to max is close to 1/2
    for v in (w.a, w.b):
        assert 0.45 < v.mean() / v.max() < 0.55


def test_ot_n1000():
    w = inputs.ot_n1000()
    assert (w.n, w.m, w.d) == (1000, 1000, 5)
    assert (w.eps, w.lam, w.tol, w.dtype) == (0.1, math.inf, 1e-6, "f64")
    assert w.s == pytest.approx(8 * 1000 * math.log(1000)) and round(w.s) == 55262
    _check_weights(w, 1.0, 1.0)
    # x ~ N(0, I), y ~ N(1, I)
    assert np.abs(w.x.mean(0)).max() < 0.12 and np.abs(w.y.mean(0) - 1.0).max() < 0.12
    assert np.abs(w.x.std(0) - 1.0).max() < 0.08


def test_uot_n20000():
    w = inputs.uot_n20000()
    assert (w.n, w.m, w.d) == (20000, 20000, 10)
    assert (w.eps, w.lam, w.tol, w.dtype) == (0.05, 1.0, 1e-5, "f32")
    assert w.s == pytest.approx(16 * 20000 * math.log(20000))
    _check_weights(w, 1.0, 1.5)
    # x: three equal components at 0 and +-4 e_1 (identity covariance): first-coordinate variance 1 + 32/3
    assert abs(w.x[:, 0].var() - (1 + 32 / 3)) < 0.5 and abs(w.x[:, 1:].var() - 1.0) < 0.05
    # y: multivariate t with 3 degrees of freedom -- heavy tails (finite variance 3, infinite kurtosis)
    r = np.linalg.norm(w.y, axis=1)
    assert np.percentile(r, 99.9) > 3 * np.percentile(r, 50)
    assert abs(np.median(np.abs(w.y)) - 0.765) < 0.03   # median |t_3| = 0.7649


@pytest.mark.parametrize("make,n,k,dtype", [(inputs.ot_n200000, 200000, 8, "bf16"),
                                           (inputs.ot_n1000000, 1000000, 16, "f32")])
def test_gaussian_mixture_workloads(make, n, k, dtype):
    w = make()
    assert (w.n, w.m, w.d) == (n, n, 3)
    assert (w.eps, w.lam, w.tol, w.dtype) == (0.01, math.inf, 1e-5, dtype)
    assert w.s == pytest.approx(16 * n * math.log(n))
    _check_weights(w, 1.0, 1.0)
    # points lie within the centre box [-5, 5]^3 grown by a few sigma = 0.5
    assert np.abs(w.x).max() < 5 + 6 * 0.5 and np.abs(w.y).max() < 5 + 6 * 0.5
    assert f"gmm{k}" in w.name


def test_frames():
    fr = inputs.frames()
    assert len(fr) == 64
    sizes = [c.shape[0] for c, _ in fr]
    assert 2000 <= min(sizes) and max(sizes) <= 9000
    assert max(sizes) > 1.5 * min(sizes)          # uneven supports
    for coords, mass in fr:
        assert coords.shape[1] == 2 and coords.min() >= 0 and coords.max() <= 95
        assert len(np.unique(coords[:, 0] * 96 + coords[:, 1])) == coords.shape[0]   # distinct pixels
        assert (mass > 0).all()
    # masses are intensities over the mean frame total: frames differ in mass
    totals = np.array([m.sum() for _, m in fr])
    assert totals.std() > 0.01 * totals.mean()
    # periodic: frames t and t + 20 have the same blob geometry (noise differs)
    assert abs(sizes[3] - sizes[23]) < 0.1 * sizes[3]
    assert len(inputs.frame_pairs()) == 64 * 63 // 2 == 2016
    assert inputs.FRAME_COST_SCALE == 2 * 95.0 ** 2


def test_budget_helpers():
    assert inputs.s_budget(1000, 8.0) == pytest.approx(8000 * math.log(1000))
    # s0(n) = 1e-3 n ln^4 n with the natural log
    assert inputs.s0(math.e ** 2) == pytest.approx(1e-3 * math.e ** 2 * 16)


def test_seeded_and_reproducible():
    a, b = inputs.uot_n20000(), inputs.uot_n20000()
    assert np.array_equal(a.x, b.x) and np.array_equal(a.b, b.b)
    c = inputs.uot_n20000(seed=3)
    assert not np.array_equal(a.x, c.x)
