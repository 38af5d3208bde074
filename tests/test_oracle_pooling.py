"""Pins of the pooling-family oracle (oracle/pooling.py) against closed forms,
library routines and hand-worked cases (Section "Spatio-temporal Aggregation
of Quality Scores")."""
import math

import numpy as np
import pytest
from scipy import stats

from oracle import pooling as P


def _rng(seed=0):
    return np.random.default_rng(seed)


def test_percentile_is_numpy_linear():
    for n in (1, 2, 5, 17, 1000):
        v = _rng(n).uniform(-0.2, 1.0, n)
        for p in (0, 6, 10, 25, 50, 75, 90, 100):
            assert P.percentile(v, p) == pytest.approx(np.percentile(v, p, method="linear"), abs=1e-15)
    # hand example: sorted (1, 2, 4, 8), p = 50: h = 1.5 -> 2 + 0.5 (4 - 2) = 3
    assert P.percentile([8, 1, 4, 2], 50) == 3.0


@pytest.mark.parametrize("c", [0.25, 0.9, -0.3])
def test_constant_map_closed_forms(c):
    q = np.full((7, 9), c)
    assert P.mean(q) == pytest.approx(c)
    assert P.cov(q) == pytest.approx(0.0, abs=1e-15)
    assert P.md(q, 2, 1) == pytest.approx(0.0, abs=1e-15)
    assert P.mink(q, 3) == pytest.approx((1 - c) ** 3)
    assert P.dw(q, 0.5) == pytest.approx(c)
    assert P.fns(q) == pytest.approx(c)
    assert P.median(q) == pytest.approx(c)
    assert P.pp(q, 10, 4) == pytest.approx(c / 4)  # every value is at the percentile
    assert P.gm_dssim(q) == pytest.approx(1 - c)
    assert P.hm_dssim(q) == pytest.approx(1 - c)


def test_two_valued_map_closed_forms():
    a, b = 0.4, 0.8
    q = np.array([a, b] * 50)
    assert P.cov(q) == pytest.approx(abs(a - b) / (a + b))      # population std |a-b|/2 over mean (a+b)/2
    assert P.md(q, 2, 1) == pytest.approx(abs(a - b) / 2)
    assert P.md(q, 1, 1) == pytest.approx(abs(a - b) / 2)
    assert P.md(q, 2, 3) == pytest.approx((abs(a - b) / 2) ** 3)
    assert P.dw(q, 1) == pytest.approx(((1 - a) * a + (1 - b) * b) / ((1 - a) + (1 - b)))
    assert P.mink(q, 2) == pytest.approx(((1 - a) ** 2 + (1 - b) ** 2) / 2)
    # lowest 10% is {a}: PP divides the a half by r
    assert P.pp(q, 10, 4) == pytest.approx((a / 4 + b) / 2)


def test_special_cases_reduce_to_the_mean():
    q = _rng(3).uniform(-0.1, 1.0, (20, 30))
    m = q.mean()
    assert P.dw(q, 0) == pytest.approx(m)          # (1-Q)^0 = 1: plain mean
    assert P.pp(q, 25, 1) == pytest.approx(m)      # r = 1: nothing reweighted
    assert P.lw(q, np.full(q.shape, 37.0), 0, 0) == pytest.approx(m)  # a = b = 0 is the baseline
    assert P.mink(q, 1) == pytest.approx(1 - m)
    s = _rng(4).uniform(0.5, 1.0, 40)
    assert P.windowed(s, 1, "am") == pytest.approx(s.mean())
    assert P.windowed(s, 1, "gm") == pytest.approx(s.mean())  # a window of one value
    assert P.windowed(s, 1, "cov") == pytest.approx(0.0, abs=1e-15)
    assert P.windowed(s, s.size, "gm") == pytest.approx(stats.gmean(s))
    assert P.windowed(s, s.size, "hm") == pytest.approx(stats.hmean(s))


def test_pythagorean_means_match_scipy_and_order():
    s = _rng(5).uniform(0.3, 1.0, 101)
    assert P.gm(s) == pytest.approx(stats.gmean(s))
    assert P.hm(s) == pytest.approx(stats.hmean(s))
    assert P.mean(s) >= P.gm(s) >= P.hm(s)
    q = _rng(6).uniform(-0.5, 0.99, 500)
    assert P.gm_dssim(q) == pytest.approx(stats.gmean(1 - q))
    assert P.hm_dssim(q) == pytest.approx(stats.hmean(1 - q))
    assert P.gm_dssim(np.array([1.0, 0.5])) == 0.0
    assert P.hm_dssim(np.array([1.0, 0.5])) == 0.0


def test_fns_of_five_values_is_their_mean():
    v = _rng(7).uniform(size=5)  # quartile positions h = 1, 2, 3 fall on order statistics
    assert P.fns(v) == pytest.approx(v.mean())
    w = np.array([0.0, 1.0, 2.0, 3.0, 4.0, 5.0, 6.0, 7.0, 8.0])  # h = 2, 4, 6
    assert P.fns(w) == pytest.approx((0 + 2 + 4 + 6 + 8) / 5)


def test_windowed_hand_example():
    s = np.array([1.0, 2.0, 4.0, 8.0])
    assert P.windowed(s, 2, "am") == pytest.approx((1.5 + 3 + 6) / 3)
    assert P.windowed(s, 2, "gm") == pytest.approx((math.sqrt(2) + math.sqrt(8) + math.sqrt(32)) / 3)
    assert P.windowed(s, 3, "hm") == pytest.approx((3 / (1 + 0.5 + 0.25) + 3 / (0.5 + 0.25 + 0.125)) / 2)
    with pytest.raises(ValueError):
        P.windowed(s, 5)


def test_luminance_weights_piecewise():
    q = np.array([0.5, 0.6, 0.7, 0.8])
    mu = np.array([5.0, 15.0, 25.0, 45.0])
    # a = 10, b = 20: weights 0, 0.25, 0.75, 1
    assert P.lw(q, mu, 10, 20) == pytest.approx((0 + 0.25 * 0.6 + 0.75 * 0.7 + 0.8) / 4)
    assert P.lw(q, mu, 10, 0) == pytest.approx((0.6 + 0.7 + 0.8) / 4)  # a step at a


def test_dw_all_perfect_is_nan():
    assert math.isnan(P.dw(np.ones(6), 1.0))


def test_local_mean_is_the_window_statistic():
    import oracle

    r = _rng(9)
    x = r.uniform(0, 255, (30, 41))
    y = r.uniform(0, 255, (30, 41))
    for kind, k, s in (("gaussian", 11, 1), ("box", 8, 4), ("gaussian", 7, 2)):
        w = oracle.window(kind, k, 1.5 if k == 11 else 1.0)
        st = oracle.window_stats(x, y, w, s)
        np.testing.assert_allclose(P.local_mean(x, w, s), st["mu1"], rtol=0, atol=1e-10)
