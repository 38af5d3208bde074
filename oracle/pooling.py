"""FP64 oracle of the pooling family (Section "Spatio-temporal Aggregation of
Quality Scores" of arXiv 2101.06354): the ways a map of local SSIM values, or
a series of frame scores, is reduced to one number.

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle``: only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py``'s oracle legs import it.

Each function writes the paper's definition out over a plain float64 array
(a map or a series alike; a map is flattened).  Order statistics use the
linear interpolation between sorted values at position h = p/100 (n-1)
(Hyndman-Fan type 7), as the temporal percentile does.  Readings of points
the paper leaves open are noted per function.  Pinned by
``tests/test_oracle_pooling.py``.
"""
from __future__ import annotations

import math

import numpy as np


def _v(a) -> np.ndarray:
    return np.asarray(a, dtype=np.float64).ravel()


def percentile(values, p: float) -> float:
    """p-th percentile, linear between the order statistics around
    h = p/100 (n-1) of the sorted values."""
    v = np.sort(_v(values))
    n = v.size
    h = p / 100.0 * (n - 1)
    lo = int(math.floor(h))
    hi = min(lo + 1, n - 1)
    return float(v[lo] + (h - lo) * (v[hi] - v[lo]))


def mean(values) -> float:
    """Arithmetic mean (the baseline MSSIM pooling)."""
    v = _v(values)
    return float(v.sum() / v.size)


def cov(values) -> float:
    """Coefficient of variation S_CoV = sigma_Q / mu_Q (Eq. of the CoV
    subsection, after MOVIE).  Reading: sigma_Q is the population standard
    deviation (divide by the number of values)."""
    v = _v(values)
    mu = v.sum() / v.size
    return float(math.sqrt(((v - mu) ** 2).sum() / v.size) / mu)


def gm_dssim(values) -> float:
    """Geometric mean of the dissimilarities 1 - Q (Moment-Based Pooling:
    the spatial GM is taken on DSSIM since local SSIM can be negative)."""
    v = 1.0 - _v(values)
    with np.errstate(divide="ignore"):
        return float(np.exp(np.log(v).sum() / v.size))


def hm_dssim(values) -> float:
    """Harmonic mean of the dissimilarities 1 - Q (as gm_dssim); a zero
    dissimilarity gives 0."""
    v = 1.0 - _v(values)
    if np.any(v == 0.0):
        return 0.0
    return float(v.size / (1.0 / v).sum())


def gm(values) -> float:
    """Geometric mean of positive values (temporal GM of frame scores)."""
    v = _v(values)
    return float(np.exp(np.log(v).sum() / v.size))


def hm(values) -> float:
    """Harmonic mean of positive values (temporal HM of frame scores)."""
    v = _v(values)
    return float(v.size / (1.0 / v).sum())


def median(values) -> float:
    """Sample median (the 50th percentile)."""
    return percentile(values, 50.0)


def fns(values) -> float:
    """Five-number summary S_FNS = (min + Q1 + median + Q3 + max) / 5."""
    return (percentile(values, 0.0) + percentile(values, 25.0) + percentile(values, 50.0) +
            percentile(values, 75.0) + percentile(values, 100.0)) / 5.0


def md(values, p: float = 2.0, o: float = 1.0) -> float:
    """Mean-deviation pooling S_MD = ((1/n sum |Q - mu_Q|^p)^(1/p))^o.
    Reading: the deviation is the Minkowski distance of order p, so the
    differences enter in absolute value."""
    v = _v(values)
    mu = v.sum() / v.size
    return float(((np.abs(v - mu) ** p).sum() / v.size) ** (1.0 / p)) ** o


def lw(values, mu_ref, a: float, b: float) -> float:
    """Luminance-weighted pooling S_LW = (1/n) sum w(mu_1) Q with
    w = 0 below a, (mu_1 - a)/b on [a, a + b), 1 from a + b on; mu_ref is the
    local mean of the reference at each map position."""
    v, m = _v(values), _v(mu_ref)
    w = np.where(m < a, 0.0, np.where(m < a + b, (m - a) / b if b > 0 else 1.0, 1.0))
    return float((w * v).sum() / v.size)


def dw(values, p: float) -> float:
    """Distortion-weighted pooling S_DW = sum (1-Q)^p Q / sum (1-Q)^p.
    All values equal to 1 give 0/0 (NaN)."""
    v = _v(values)
    wt = (1.0 - v) ** p
    with np.errstate(invalid="ignore", divide="ignore"):
        return float((wt * v).sum() / wt.sum())


def mink(values, p: float) -> float:
    """Minkowski pooling of the dissimilarities, S_Mink = (1/n) sum (1-Q)^p."""
    v = _v(values)
    return float(((1.0 - v) ** p).sum() / v.size)


def pp(values, p: float, r: float) -> float:
    """Percentile pooling: values at or below the p-th percentile are divided
    by r, then everything is averaged."""
    v = _v(values)
    t = percentile(v, p)
    return float(np.where(v <= t, v / r, v).sum() / v.size)


def windowed(values, k: int, kind: str = "am") -> float:
    """Windowed temporal pooling (Moment-Based Pooling): the mean of a
    per-window statistic over the windows of k consecutive values.  Reading:
    the windows are the n - k + 1 full windows [t, t + k); kind is 'am', 'gm',
    'hm' or 'cov' (W-AM, W-GM, W-HM, W-CoV)."""
    v = _v(values)
    n = v.size
    if not 1 <= k <= n:
        raise ValueError("window size must be in 1..n")
    f = {"am": mean, "gm": gm, "hm": hm, "cov": cov}[kind]
    return float(sum(f(v[t:t + k]) for t in range(n - k + 1)) / (n - k + 1))


def local_mean(img, w, stride: int = 1):
    """Window-weighted local mean mu(i, j) = sum_{m,n} w(m, n) img(i s + m, j s + n)
    at every valid strided position (Eq. local_means): the mu_1 map that
    luminance-weighted pooling weights by."""
    a = np.asarray(img, dtype=np.float64)
    k = w.shape[0]
    oh = (a.shape[0] - k) // stride + 1
    ow = (a.shape[1] - k) // stride + 1
    out = np.zeros((oh, ow))
    for m in range(k):
        for n in range(k):
            out += w[m, n] * a[m:m + stride * (oh - 1) + 1:stride, n:n + stride * (ow - 1) + 1:stride]
    return out
