"""Pin of the dense iterations and the objective (Alg. 1 and the output line
of Alg. 3) against the closed form of entropic OT between Gaussian measures.

The oracle solves min <T, C> - eps H(T), H(T) = -sum T (log T - 1), over
couplings of the discrete marginals mu, nu.  With the marginals fixed,
    <T, C> + eps KL(T | mu x nu) = <T, C> - eps H(T) + eps + eps (H(mu) + H(nu)),
H(mu) = -sum mu log mu, so both problems have the same minimiser and values
that differ by that constant.  Gaussians sampled on a uniform grid fine
against their widths (masses proportional to the density) give discrete
problems whose KL-regularised value converges very fast to the value for the
continuous Gaussians, which has a closed form:

- d = 1, N(m1, a^2) and N(m2, b^2), cost |x - y|^2: the optimal coupling is
  Gaussian; with covariance c between the two coordinates its cost is
  (m1 - m2)^2 + a^2 + b^2 - 2c and its KL to the product is
  -log(1 - c^2 / (a^2 b^2)) / 2.  Setting the derivative in c to zero gives
  2 c^2 + eps c - 2 a^2 b^2 = 0, so c = (sqrt(eps^2 + 16 a^2 b^2) - eps) / 4.
- any d, N(m1, A) and N(m2, B) (Janati, Muzellec, Peyre and Cuturi, NeurIPS
  2020; Mallasto et al. 2021): with s = eps / 2 and
  D = (4 A^{1/2} B A^{1/2} + s^2 I)^{1/2},
  value = |m1 - m2|^2 + tr A + tr B - tr D + d s (1 - log 2s) + s log det(D + s I).
  The two forms agree at d = 1, which the test checks first.
"""
import math

import numpy as np
import pytest
from scipy import linalg


def _closed_1d(m1, a, m2, b, eps):
    c = (math.sqrt(eps * eps + 16 * a * a * b * b) - eps) / 4
    return (m1 - m2) ** 2 + a * a + b * b - 2 * c - eps / 2 * math.log(1 - c * c / (a * a * b * b))


def _closed(m1, A, m2, B, eps):
    d = len(m1)
    s = eps / 2
    Ah = linalg.sqrtm(A).real
    D = linalg.sqrtm(4 * Ah @ B @ Ah + s * s * np.eye(d)).real
    return float(((m1 - m2) ** 2).sum() + np.trace(A) + np.trace(B) - np.trace(D)
                 + d * s * (1 - math.log(2 * s)) + s * math.log(np.linalg.det(D + s * np.eye(d))))


def _density(g, m, S):
    z = g - m
    w = np.exp(-0.5 * np.einsum("ki,ij,kj->k", z, np.linalg.inv(S), z))
    return w / w.sum()


def _kl_value(orc, g, m1, A, m2, B, eps, log_domain):
    mu, nu = _density(g, m1, A), _density(g, m2, B)
    kx, ky = mu > 1e-200, nu > 1e-200       # grid points with (numerically) no mass are left out
    x, y, mu, nu = g[kx], g[ky], mu[kx], nu[ky]
    P = orc.OracleProblem(mu, nu, eps, 1.0, math.inf, x=x, y=y, cost_norm=0)
    r = orc.dense_sinkhorn(P, tol=1e-12, max_iter=100000, log_domain=log_domain)
    assert r["info"]["status"] == 0
    ent = -(mu * np.log(mu)).sum() - (nu * np.log(nu)).sum()
    return r["obj"] + eps + eps * ent


def test_closed_forms_agree_in_one_dimension():
    for m1, a, m2, b, eps in [(0.0, 1.0, 1.5, 0.6, 0.2), (0.3, 0.8, -0.4, 1.3, 0.05)]:
        ref = _closed(np.array([m1]), np.array([[a * a]]), np.array([m2]), np.array([[b * b]]), eps)
        assert _closed_1d(m1, a, m2, b, eps) == pytest.approx(ref, rel=1e-13)


@pytest.mark.parametrize("m1,a,m2,b,eps", [(0.0, 1.0, 1.5, 0.6, 0.2), (0.3, 0.8, -0.4, 1.3, 0.05)])
def test_one_dimensional_gaussians(orc, m1, a, m2, b, eps):
    h, L = 0.08, 7.0
    g = np.arange(min(m1 - L * a, m2 - L * b), max(m1 + L * a, m2 + L * b) + h / 2, h)[:, None]
    v = _kl_value(orc, g, np.array([m1]), np.array([[a * a]]), np.array([m2]), np.array([[b * b]]), eps,
                  log_domain=eps < 0.1)
    assert v == pytest.approx(_closed_1d(m1, a, m2, b, eps), rel=2e-8)


def _rot(t):
    return np.array([[math.cos(t), -math.sin(t)], [math.sin(t), math.cos(t)]])


@pytest.mark.parametrize("eps", [0.5, 0.25])
def test_two_dimensional_correlated_gaussians(orc, eps):
    A = _rot(0.4) @ np.diag([1.0, 0.36]) @ _rot(0.4).T
    B = _rot(-0.9) @ np.diag([0.64, 1.21]) @ _rot(-0.9).T
    m1, m2 = np.array([0.2, -0.3]), np.array([-0.5, 0.6])
    t = np.arange(-6.4, 6.4 + 0.2, 0.4)
    g = np.stack(np.meshgrid(t, t, indexing="ij"), -1).reshape(-1, 2)
    v = _kl_value(orc, g, m1, A, m2, B, eps, log_domain=False)
    assert v == pytest.approx(_closed(m1, A, m2, B, eps), rel=2e-8)
