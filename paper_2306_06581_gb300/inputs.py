"""Seeded synthetic inputs shaped like the paper's workloads.

This module only draws random points and weights (numpy, seeded) and states
the parameters of each workload; it performs none of the method's
arithmetic, so both the CUDA path and the CPU oracle can take their inputs
from it.

Workloads (sizes follow the five configurations this library is measured on):
  ot_n1000     balanced OT, n=m=1000 in R^5, x~N(0,I), y~N(1,I), a,b~U(0,1)
               normalised, eps=0.1, s=8 n ln n, FP64, tol 1e-6
  uot_n20000   UOT lambda=1, n=m=20000 in R^10, x from a 3-component
               Gaussian mixture, y multivariate t (nu=3), |a|=1, |b|=1.5,
               eps=0.05, s=16 n ln n, FP32, tol 1e-5
  ot_n200000   balanced OT, n=m=2e5 in R^3, 8-component Gaussian mixtures,
               eps=0.01 (log-domain absorption), s=16 n ln n
  frames_uot   64 synthetic 96x96 frames (two pulsing Gaussian blobs, period
               20 frames, 5% noise), supports thresholded to 2k-9k pixels,
               all 2016 pairs as UOT lambda=1, eps=0.01
  ot_n1000000  balanced OT, n=m=1e6 in R^3, 16-component Gaussian mixtures,
               eps=0.01, s=16 n ln n, FP32, tol 1e-5
The cost is the squared Euclidean distance divided by its maximum over all
pairs (section 5.1 uses squared Euclidean cost; the normalisation makes
eps comparable across workloads).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Workload:
    name: str
    x: np.ndarray          # n x d, float64
    y: np.ndarray          # m x d, float64
    a: np.ndarray          # n, float64
    b: np.ndarray          # m, float64
    eps: float
    lam: float             # math.inf: balanced OT
    s: float               # expected sample budget
    tol: float
    dtype: str             # value / iterate precision of the workload
    seed: int = 0x5EED     # Philox seed of the sampling stream
    pid: int = 0
    extra: dict = field(default_factory=dict)

    @property
    def n(self):
        return self.a.size

    @property
    def m(self):
        return self.b.size

    @property
    def d(self):
        return self.x.shape[1]


def s_budget(n: int, factor: float) -> float:
    """s = factor * n * ln n (natural log)."""
    return float(factor * n * math.log(n))


def s0(n: float) -> float:
    """The paper's reference budget s0(n) = 1e-3 n log^4 n (section 5.1), natural log."""
    return 1e-3 * n * math.log(n) ** 4


def _uniform_weights(rng, n, total=1.0):
    w = rng.uniform(0.0, 1.0, n)
    return w * (total / w.sum())


def _gmm(rng, n, d, centres, sigma, weights):
    comp = rng.choice(len(weights), size=n, p=weights)
    return centres[comp] + sigma * rng.standard_normal((n, d))


def small_problem(n=64, m=None, d=3, seed=0, eps=0.1, lam=math.inf, s_factor=8.0, mass_a=1.0,
                  mass_b=1.0, shift=1.0, dtype="f64"):
    """A small random problem for tests: x~N(0,I), y~N(shift,I), U(0,1) weights."""
    m = n if m is None else m
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((n, d))
    y = rng.standard_normal((m, d)) + shift
    a = _uniform_weights(rng, n, mass_a)
    b = _uniform_weights(rng, m, mass_b)
    return Workload(f"small_n{n}_m{m}_d{d}", x, y, a, b, eps, lam, s_budget(max(n, 2), s_factor),
                    1e-6, dtype, seed=0x5EED + seed)


def ot_n1000(seed=1, n=1000):
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((n, 5))
    y = rng.standard_normal((n, 5)) + 1.0
    a = _uniform_weights(rng, n)
    b = _uniform_weights(rng, n)
    return Workload(f"ot_n{n}_d5_eps0.1_f64", x, y, a, b, 0.1, math.inf, s_budget(n, 8.0), 1e-6,
                    "f64")


def uot_n20000(seed=2, n=20000):
    rng = np.random.default_rng(seed)
    d = 10
    centres = np.zeros((3, d))
    centres[1, 0], centres[2, 0] = 4.0, -4.0
    x = _gmm(rng, n, d, centres, 1.0, np.full(3, 1.0 / 3.0))
    z = rng.standard_normal((n, d))
    w = rng.chisquare(3.0, n)
    y = z / np.sqrt(w / 3.0)[:, None]
    a = _uniform_weights(rng, n, 1.0)
    b = _uniform_weights(rng, n, 1.5)
    return Workload(f"uot_n{n}_d10_lam1_eps0.05_f32", x, y, a, b, 0.05, 1.0, s_budget(n, 16.0),
                    1e-5, "f32")


def ot_gmm(n, d=3, k=8, seed=3, eps=0.01, s_factor=16.0, tol=1e-5, dtype="f32", name=None):
    rng = np.random.default_rng(seed)
    cx = rng.uniform(-5.0, 5.0, (k, d))
    cy = rng.uniform(-5.0, 5.0, (k, d))
    wx = rng.dirichlet(np.ones(k))
    wy = rng.dirichlet(np.ones(k))
    x = _gmm(rng, n, d, cx, 0.5, wx)
    y = _gmm(rng, n, d, cy, 0.5, wy)
    a = _uniform_weights(rng, n)
    b = _uniform_weights(rng, n)
    return Workload(name or f"ot_n{n}_d{d}_gmm{k}_eps{eps}", x, y, a, b, eps, math.inf,
                    s_budget(n, s_factor), tol, dtype)


def ot_n200000(seed=3, n=200000, dtype="bf16"):
    return ot_gmm(n, 3, 8, seed, 0.01, 16.0, 1e-5, dtype, name=f"ot_n{n}_d3_gmm8_eps0.01_{dtype}")


def ot_n1000000(seed=5, n=1000000):
    return ot_gmm(n, 3, 16, seed, 0.01, 16.0, 1e-5, "f32", name=f"ot_n{n}_d3_gmm16_eps0.01_f32")


def frames(seed=4, n_frames=64, size=96, period=20.0, noise=0.05):
    """Synthetic periodic image sequence: two Gaussian blobs whose radius and
    centre vary sinusoidally with the given period, plus uniform noise on 5%
    of the pixels.  Returns a list of (coords[k,2], mass[k]) supports after
    thresholding each frame to its brightest pixels (2k-9k per frame)."""
    rng = np.random.default_rng(seed)
    yy, xx = np.mgrid[0:size, 0:size].astype(np.float64)
    out = []
    raw = []
    for t in range(n_frames):
        ph = 2.0 * math.pi * t / period
        r0 = 18.0 * (1.0 + 0.5 * math.sin(ph))
        r1 = 12.0 * (1.0 + 0.5 * math.cos(ph))
        c0 = (32.0 + 10.0 * math.sin(ph), 40.0 + 6.0 * math.cos(ph))
        c1 = (64.0 + 8.0 * math.cos(ph), 56.0 + 10.0 * math.sin(ph))
        img = np.exp(-((xx - c0[0]) ** 2 + (yy - c0[1]) ** 2) / (2 * r0 ** 2))
        img += 0.8 * np.exp(-((xx - c1[0]) ** 2 + (yy - c1[1]) ** 2) / (2 * r1 ** 2))
        mask = rng.uniform(size=img.shape) < noise
        img = img + mask * rng.uniform(0.0, 0.3, img.shape)
        raw.append(img)
    mean_total = float(np.mean([im.sum() for im in raw]))
    for img in raw:
        thr = np.quantile(img, 1.0 - _support_fraction(img))
        keep = img > thr
        ys, xs = np.nonzero(keep)
        coords = np.stack([xs, ys], axis=1).astype(np.float64)
        out.append((coords, img[keep] / mean_total))
    return out


def _support_fraction(img):
    # a frame keeps its pixels above 12% of its own peak, clipped so that the
    # support holds between 2000 and 9000 pixels
    k = int(np.count_nonzero(img > 0.12 * img.max()))
    k = min(max(k, 2000), 9000)
    return k / img.size


def frame_pairs(n_frames=64):
    return [(i, j) for i in range(n_frames) for j in range(i + 1, n_frames)]


FRAME_COST_SCALE = 2.0 * 95.0 ** 2   # squared pixel distance / (2 * 95^2)


WORKLOADS = {
    "ot_n1000": ot_n1000,
    "uot_n20000": uot_n20000,
    "ot_n200000": ot_n200000,
    "ot_n1000000": ot_n1000000,
}


def mlp_weights(d, seed, scale=1.0):
    """Seeded warm-start network weights that are exact in BF16 (k / 2^10 with
    |k| <= 255, times a power-of-two scale), for checks that feed the same
    weights to the GPU and to the CPU reference.  Both sides, source first."""
    rng = np.random.default_rng(seed)
    F, E, H = d + 1, 16, 128
    D0 = F + E
    sizes = [E * F, E, H * D0, H, H * H, H, H, 1]
    fans = [F, 0, D0, 0, H, 0, H, 0]
    out = []
    for _ in range(2):
        for sz, fan in zip(sizes, fans):
            lim = math.sqrt(6.0 / fan) if fan else 0.05
            k = np.clip(np.rint(rng.uniform(-lim, lim, sz) * 1024.0 * scale), -255, 255)
            out.append(k / 1024.0)
    return np.concatenate(out)


def ot_gmm16(n, seed, eps=0.01):
    """The 16-component mixture family in R^3 (balanced OT, s = 16 n ln n)."""
    return ot_gmm(n, 3, 16, seed, eps, 16.0, 1e-5, "f32", name=f"ot_n{n}_d3_gmm16_seed{seed}")


def ibp_measures(n):
    """The synthetic barycenter recipe of the paper's appendix on a 1-D grid of
    n points (i + 0.5) / n: a Gaussian N(0.2, 1/50), an equal mixture of
    N(0.5, 1/60) and N(0.8, 1/80), and a t density with 5 degrees of freedom
    at 0.6 with scale sqrt(1/100); each plus 1e-2 of its maximum, normalised.
    Returns (grid points n x 1, [b_1, b_2, b_3])."""
    from scipy import stats
    g = (np.arange(n) + 0.5) / n
    b1 = stats.norm.pdf(g, 0.2, math.sqrt(1 / 50))
    b2 = 0.5 * stats.norm.pdf(g, 0.5, math.sqrt(1 / 60)) + 0.5 * stats.norm.pdf(g, 0.8, math.sqrt(1 / 80))
    b3 = stats.t.pdf((g - 0.6) / math.sqrt(1 / 100), 5)
    out = []
    for b in (b1, b2, b3):
        b = b + 1e-2 * b.max()
        out.append(b / b.sum())
    return g.reshape(-1, 1), out
