"""Pins for the oracle's binary32 exp / log (used by the UOT sampling
decision of Eq. pij-uot) and its exact summation, against libm in FP64 and
Python's correctly rounded math.fsum."""
import math

import numpy as np


def _ulp_err(got32, ref64):
    got = got32.astype(np.float64)
    ulp = np.spacing(np.abs(ref64).astype(np.float32)).astype(np.float64)
    return np.abs(got - ref64) / ulp


def test_exp32_error_bound(orc):
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.uniform(-103.0, 88.7, 200000), rng.uniform(-1, 1, 50000),
                        np.linspace(-87.3, 88.7, 10001)]).astype(np.float32)
    ref = np.exp(x.astype(np.float64))
    normal = ref > 1.2e-38
    err = _ulp_err(orc.exp32(x)[normal], ref[normal])
    assert err.max() <= 2.0, err.max()
    # subnormal range: absolute error within a couple of subnormal steps
    sub = ~normal
    assert np.abs(orc.exp32(x)[sub].astype(np.float64) - ref[sub]).max() <= 2 * 2.0 ** -149


def test_exp32_special_values(orc):
    x = np.array([0.0, -0.0, 1.0, -1.0, 100.0, -200.0, np.inf, -np.inf, np.nan], np.float32)
    y = orc.exp32(x)
    assert y[0] == 1.0 and y[1] == 1.0
    assert abs(y[2] - math.e) < 1e-6 and abs(y[3] - 1 / math.e) < 1e-7
    assert np.isinf(y[4]) and y[5] == 0.0 and np.isinf(y[6]) and y[7] == 0.0 and np.isnan(y[8])
    # monotone and never above 1 on [-1, 0] (the range of the UOT weight factor)
    t = np.linspace(-1.0, 0.0, 100001).astype(np.float32)
    e = orc.exp32(t)
    assert (np.diff(e.astype(np.float64)) >= 0).all() and e.max() <= 1.0


def test_log32_error_bound(orc):
    rng = np.random.default_rng(1)
    x = np.concatenate([
        np.exp(rng.uniform(-87, 88, 200000)),
        rng.uniform(0.5, 2.0, 50000),
        np.array([1e-45, 1e-40, 3e-39, 1.1754942e-38, 1.0, 2.0, 0.5, 3.4e38]),
    ]).astype(np.float32)
    x = x[x > 0]
    ref = np.log(x.astype(np.float64))
    got = orc.log32(x).astype(np.float64)
    # absolute error relative to the ulp of the result, floor at 2^-24 near log(1)=0
    ulp = np.maximum(np.spacing(np.abs(ref).astype(np.float32)).astype(np.float64), 2.0 ** -24)
    assert (np.abs(got - ref) / ulp).max() <= 2.0
    assert orc.log32(np.array([1.0], np.float32))[0] == 0.0
    assert orc.log32(np.array([0.0], np.float32))[0] == -np.inf


def test_exact_sum_matches_fsum(orc):
    rng = np.random.default_rng(2)
    cases = [
        rng.uniform(0, 1, 100000),
        np.exp(rng.uniform(-100, 80, 50000)),
        np.concatenate([np.full(1000, 3.4e38 / 4096), np.full(1000, 1e-45), rng.uniform(0, 1e-38, 1000)]),
        np.full(300000, 16777215.0),           # many equal values: digit carries
        np.array([1.0, 2.0 ** -149, 2.0 ** -60, 2.0 ** 53]),
        np.array([0.0, 0.0]),
        np.array([], dtype=np.float64),
    ]
    for c in cases:
        x = np.asarray(c).astype(np.float32)
        assert orc.exact_sum_f32(x) == math.fsum(x.astype(np.float64).tolist())


def test_exact_sum_rounding_at_ties(orc):
    # sums that land exactly halfway between two doubles, or just beyond it
    # with the only extra bit one or many places below the rounding bit:
    # fsum rounds to nearest, ties to even
    u = 2.0 ** -52
    cases = [
        [1.0, u / 2],                         # tie, even neighbour below: stays 1
        [1.0, u, u / 2],                      # tie, odd mantissa: rounds up to 1 + 2u
        [1.0, u / 2, u / 4],                  # above the tie by the next bit: rounds up
        [1.0, u / 2, 2.0 ** -149],            # above the tie by the smallest subnormal: rounds up
        # 2^53 - 1 + 1/2: a tie whose rounding carries into the next binade
        [2.0 ** 52, 2.0 ** 52 - 2.0 ** 28, 2.0 ** 28 - 16, 15.0, 0.5],
        [2.0 ** 100, 2.0 ** 47],              # tie far above 1
        [2.0 ** 100, 2.0 ** 48, 2.0 ** 47],
    ]
    for c in cases:
        x = np.array(c, np.float64).astype(np.float32)
        assert np.array_equal(x.astype(np.float64), np.array(c)), c     # every term is a binary32
        assert orc.exact_sum_f32(x) == math.fsum(c), c
    rng = np.random.default_rng(5)
    ties = 0
    for _ in range(3000):
        # 1 plus multiples of 2^-60: the bits below the double's last one are often all zero
        k = rng.integers(0, 1 << 10, 3)
        c = [1.0] + [float(v) * 2.0 ** -60 for v in k]
        ties += (int(sum(k)) & 0x7F) == 0x40
        assert orc.exact_sum_f32(np.array(c, np.float32)) == math.fsum(c)
    assert ties > 5


def test_exact_sum_order_independent(orc):
    rng = np.random.default_rng(3)
    x = np.exp(rng.uniform(-60, 20, 20001)).astype(np.float32)
    s0 = orc.exact_sum_f32(x)
    for _ in range(3):
        assert orc.exact_sum_f32(rng.permutation(x)) == s0
    # a sequential float64 sum differs in general; the exact one does not depend on it
    assert abs(s0 - float(np.sum(x.astype(np.float64)))) <= 1e-12 * s0


def test_exact_sum_ties_to_even(orc):
    # 2^53 + 1 is a tie between 2^53 and 2^53 + 2: rounds to even (2^53)
    x = np.array([2.0 ** 53, 1.0], np.float32)
    assert orc.exact_sum_f32(x) == 2.0 ** 53
    x = np.array([2.0 ** 53, 1.0, 2.0 ** -20], np.float32)   # sticky bit breaks the tie upwards
    assert orc.exact_sum_f32(x) == 2.0 ** 53 + 2
