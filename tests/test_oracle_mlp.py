"""Pins for the warm-start network's CPU reference (oracle/mlp_oracle.py):
- the analytic gradient equals central finite differences of the loss (FP64);
- the gauge fix keeps alpha_i + beta_j and balances sum a alpha = sum b beta;
- Adam under a constant gradient moves every weight by lr g / (|g| + eps) per step;
- the predictions do not change when all points are scaled by c and the cost
  maximum by c^2, nor when every point of either side is split into two equal
  halves (the mass features n a_i and the pooled mean see the same values);
- a network with constant output c has loss = the a-weighted mean of
  (c - target)^2 over eps^2, minimised at the weighted mean of the finite
  targets with the weighted variance over eps^2 as its value;
- the parameter count equals the library's."""
import ctypes
import math

import numpy as np
import pytest

from oracle import mlp_oracle as M
from paper_2306_06581_gb300 import inputs


def _tiny(seed=0, d=3, n=9, m=7):
    rng = np.random.default_rng(seed)
    x = rng.normal(0, 1, (n, d)); y = rng.normal(0.5, 1, (m, d))
    a = rng.uniform(0.2, 1, n); a /= a.sum()
    b = rng.uniform(0.2, 1, m); b /= b.sum()
    cm = float(((x[:, None] - y[None]) ** 2).sum(-1).max())
    ta = rng.normal(0, 0.05, n); tb = rng.normal(0, 0.05, m)
    ta[2] = -np.inf   # an unreachable row is left out of the loss
    return x, a, y, b, cm, ta, tb


def test_gradient_matches_finite_differences():
    d = 3
    x, a, y, b, cm, ta, tb = _tiny()
    rng = np.random.default_rng(1)
    w = rng.normal(0, 0.3, M.count(d))
    eps = 0.05
    L0, g = M.loss_grad(w, d, x, a, y, b, cm, ta, tb, eps)
    assert np.isfinite(L0) and g.shape == w.shape
    n1 = M.layout(d)["size"]
    o = M.layout(d)
    # every parameter group of both sides, a few coordinates each
    idx = []
    for side in (0, n1):
        for nm in ("We", "ce", "W1", "b1", "W2", "b2", "w3", "b3"):
            s0, sz = o[nm]
            idx += list(side + s0 + rng.choice(sz, min(sz, 6), replace=False))
    h = 1e-6
    for k in idx:
        wp = w.copy(); wp[k] += h
        wm = w.copy(); wm[k] -= h
        fd = (M.loss_grad(wp, d, x, a, y, b, cm, ta, tb, eps)[0] - M.loss_grad(wm, d, x, a, y, b, cm, ta, tb, eps)[0]) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * max(1.0, abs(fd)) + 1e-8, (k, fd, g[k])


def test_loss_is_zero_at_the_prediction():
    d = 2
    x, a, y, b, cm, _, _ = _tiny(3, d=d)
    w = np.random.default_rng(4).normal(0, 0.2, M.count(d))
    al, be = M.predict(w, d, x, a, y, b, cm)
    L, g = M.loss_grad(w, d, x, a, y, b, cm, al, be, 0.1)
    assert L == 0.0 and not g.any()


def test_predictions_invariant_to_scale_and_splitting():
    d = 3
    x, a, y, b, cm, _, _ = _tiny(6, d=d, n=11, m=8)
    w = np.random.default_rng(7).normal(0, 0.3, M.count(d))
    al, be = M.predict(w, d, x, a, y, b, cm)
    c = 3.7
    al2, be2 = M.predict(w, d, c * x, a, c * y, b, c * c * cm)
    assert np.allclose(al2, al, rtol=1e-12, atol=1e-13) and np.allclose(be2, be, rtol=1e-12, atol=1e-13)
    # every target point split in two halves: the source side's predictions stay
    al3, be3 = M.predict(w, d, x, a, np.repeat(y, 2, 0), np.repeat(b / 2, 2), cm)
    assert np.allclose(al3, al, rtol=1e-12, atol=1e-13)
    assert np.allclose(be3, np.repeat(be, 2), rtol=1e-12, atol=1e-13)
    # and every source point split: each copy predicts what the original did
    al4, be4 = M.predict(w, d, np.repeat(x, 2, 0), np.repeat(a / 2, 2), y, b, cm)
    assert np.allclose(al4, np.repeat(al, 2), rtol=1e-12, atol=1e-13)
    assert np.allclose(be4, be, rtol=1e-12, atol=1e-13)
    # the predictions do depend on the masses (the features are not constant)
    al5, _ = M.predict(w, d, x, np.roll(a, 1), y, b, cm)
    assert np.abs(al5 - al).max() > 1e-6


def test_constant_network_loss_is_weighted_variance():
    d = 2
    x, a, y, b, cm, ta, tb = _tiny(8, d=d)
    eps = 0.07
    o = M.layout(d)
    n1, k3 = o["size"], o["b3"][0]
    fa, fb = np.isfinite(ta), np.isfinite(tb)
    ma, mb = np.average(ta[fa], weights=a[fa]), np.average(tb[fb], weights=b[fb])
    va = np.cov(ta[fa], aweights=a[fa], bias=True)
    vb = np.cov(tb[fb], aweights=b[fb], bias=True)

    def loss(c_alpha):
        w = np.zeros(M.count(d))          # every layer zero: both outputs are their bias b3
        w[k3], w[n1 + k3] = c_alpha, mb
        return M.loss_grad(w, d, x, a, y, b, cm, ta, tb, eps)[0]

    assert loss(ma) == pytest.approx((va + vb) / eps ** 2, rel=1e-12)
    for h in (0.01, 0.1):
        # symmetric about the weighted mean, and above the minimum by h^2 / eps^2
        assert loss(ma - h) == pytest.approx(loss(ma + h), rel=1e-12)
        assert loss(ma + h) - loss(ma) == pytest.approx(h * h / eps ** 2, rel=1e-9)


def test_gauge_fix():
    rng = np.random.default_rng(5)
    a = rng.uniform(0.1, 1, 8); a /= a.sum()
    b = rng.uniform(0.1, 1, 6); b /= b.sum()
    al = rng.normal(0, 1, 8); be = rng.normal(0, 1, 6)
    al[3] = -np.inf
    a2, b2 = M.gauge_fix(a, al, b, be)
    fa = np.isfinite(al)
    assert np.allclose((a2[:, None] + b2[None])[fa], (al[:, None] + be[None])[fa], atol=1e-14)
    assert abs((a[fa] * a2[fa]).sum() - (b * b2).sum()) < 1e-14
    assert np.isneginf(a2[3])


def test_adam_constant_gradient_closed_form():
    w0 = np.array([0.5, -1.0, 2.0]); g = np.array([0.3, -0.02, 0.0])
    lr, eps = 1e-2, 1e-8
    w, m1, m2 = w0.copy(), np.zeros(3), np.zeros(3)
    for t in range(1, 11):
        w, m1, m2 = M.adam(w, m1, m2, g, t, lr, eps=eps)
    step = lr * np.abs(g) / (np.abs(g) + eps)
    assert np.allclose(w, w0 - 10 * np.sign(g) * step, rtol=0, atol=1e-12)


def test_param_count_and_bf16_exact_weights():
    d = 3
    w = inputs.mlp_weights(d, 7)
    assert w.size == M.count(d)
    # k / 2^10 with |k| <= 255: 8 significant bits, exact in BF16
    assert np.array_equal(np.rint(w * 1024), w * 1024) and np.abs(w * 1024).max() <= 255
    import os
    so = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2306_06581_gb300",
                      "libsparsink.so")
    if not os.path.exists(so):
        pytest.skip("library not built")
    L = ctypes.CDLL(so)
    L.sps_mlp_param_count.restype = ctypes.c_size_t
    assert L.sps_mlp_param_count(d) == M.count(d)
    assert L.sps_mlp_param_count(0) == 0
