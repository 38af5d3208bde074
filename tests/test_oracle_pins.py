"""Pins for the FP64 oracle against what the paper and mathematics fix.

Each test checks the oracle against something other than itself: a closed
form derived from the Background-section definitions, an invariant the paper
states (symmetry, boundedness, unique maximum), a library routine on small
inputs (scipy's 2-D correlation, numpy sliding windows / percentiles), the
paper's own integral-image identity, or central finite differences.  The
inputs are chosen so that a dropped term, a wrong sign or index, or a
transposed operand fails at least one of them.
"""
import math
import os

import numpy as np
import pytest
import scipy.signal

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "closed_forms.txt")


def _rng(seed):
    return np.random.default_rng(seed)


# --------------------------------------------------------------------------- windows

@pytest.mark.parametrize("k,sigma", [(11, 1.5), (7, 1.0), (9, 2.5), (3, 0.7)])
def test_gaussian_window_is_normalised_separable_gaussian(k, sigma):
    w = oracle.gaussian_window(k, sigma)
    assert abs(w.sum() - 1.0) < 1e-15
    np.testing.assert_array_equal(w, w.T)
    np.testing.assert_array_equal(w, w[::-1, ::-1])
    g = scipy.signal.windows.gaussian(k, std=sigma)  # library routine, independent route
    ref = np.outer(g, g) / np.outer(g, g).sum()
    np.testing.assert_allclose(w, ref, rtol=1e-13, atol=0)


def test_gaussian_taps_k11_sigma15_values():
    # normalised 1-D marginal of the recommended window (Background section)
    g = oracle.gaussian_window(11, 1.5).sum(axis=1)
    expect = [0.00102838, 0.00759876, 0.03600077, 0.10936069, 0.21300554, 0.26601172]
    np.testing.assert_allclose(g[:6], expect, atol=5e-9)
    np.testing.assert_allclose(g[5:], expect[::-1], atol=5e-9)


def test_box_window():
    w = oracle.box_window(8)
    assert w.shape == (8, 8) and np.all(w == 1 / 64)


def test_window_size_helpers():
    assert oracle.gaussian_k_for_sigma(1.5) == 11
    assert oracle.gaussian_k_for_sigma(1.0) == 7
    assert oracle.gaussian_k_for_sigma(6.0) == 43
    assert oracle.rect_k_equivalent(1.5, "variance") == 7   # K = ceil(1.5 sqrt 3) = 3
    assert oracle.rect_k_equivalent(1.5, "bandwidth") == 7  # K = ceil(2.403) = 3
    assert oracle.rect_k_equivalent(3.0, "variance") == 13  # K = ceil(5.196) = 6
    assert oracle.rect_k_equivalent(3.0, "bandwidth") == 11  # K = ceil(4.806) = 5


# --------------------------------------------------------------------------- statistics

@pytest.mark.parametrize("shape,k,s", [((13, 17), 5, 1), ((13, 17), 5, 2), ((20, 9), 4, 3),
                                       ((6, 6), 6, 1), ((11, 30), 3, 5)])
def test_window_stats_match_scipy_correlation(shape, k, s):
    r = _rng(1)
    x = r.uniform(0, 255, shape)
    y = r.uniform(0, 255, shape)
    w = r.uniform(0.1, 1.0, (k, k))  # non-symmetric on purpose: a flipped/transposed window fails
    w /= w.sum()
    st = oracle.window_stats(x, y, w, s)
    cor = lambda a: scipy.signal.correlate2d(a, w, mode="valid")[::s, ::s]
    mu1, mu2 = cor(x), cor(y)
    np.testing.assert_allclose(st["mu1"], mu1, rtol=1e-13)
    np.testing.assert_allclose(st["mu2"], mu2, rtol=1e-13)
    np.testing.assert_allclose(st["var1"], cor(x * x) - mu1 ** 2, atol=1e-8)
    np.testing.assert_allclose(st["var2"], cor(y * y) - mu2 ** 2, atol=1e-8)
    np.testing.assert_allclose(st["cov"], cor(x * y) - mu1 * mu2, atol=1e-8)


@pytest.mark.parametrize("shape,k,s", [((13, 17), 5, 1), ((20, 9), 4, 3), ((11, 30), 3, 5), ((40, 33), 11, 1)])
def test_separable_stats_match_scipy_and_direct_mode(shape, k, s):
    """The row-then-column mode (the one the CPU baseline times) against
    scipy's 2-D correlation with the outer-product window and against the
    direct k x k mode.  The 1-D factor is not symmetric, so a flipped factor
    fails, and the image is not square, so swapped passes fail."""
    r = _rng(3)
    x = r.uniform(0, 255, shape)
    y = r.uniform(0, 255, shape)
    g = r.uniform(0.1, 1.0, k)
    g /= g.sum()
    w = np.outer(g, g)
    sep = oracle.window_stats_separable(x, y, g, s)
    direct = oracle.window_stats(x, y, w, s)
    cor = lambda a: scipy.signal.correlate2d(a, w, mode="valid")[::s, ::s]
    mu1, mu2 = cor(x), cor(y)
    np.testing.assert_allclose(sep["mu1"], mu1, rtol=1e-13)
    np.testing.assert_allclose(sep["mu2"], mu2, rtol=1e-13)
    np.testing.assert_allclose(sep["cov"], cor(x * y) - mu1 * mu2, atol=1e-8)
    for key in ("mu1", "mu2", "var1", "var2", "cov"):
        np.testing.assert_allclose(sep[key], direct[key], rtol=0, atol=1e-12 * 255.0 ** 2)


def test_separable_mode_msssim_equals_direct_mode():
    """MS-SSIM through the separable mode equals the direct mode to 1e-12 on a
    smooth-noise pair (Gaussian window) and on a box-window pair."""
    r = _rng(4)
    x = np.round(r.uniform(0, 255, (180, 200)))
    y = np.clip(x + np.round(r.normal(0, 12, x.shape)), 0, 255)
    for kw in ({}, dict(window_kind="box", k=8)):
        a, pa = oracle.msssim(x, y, **kw)
        b, pb = oracle.msssim(x, y, mode="separable", **kw)
        assert abs(a - b) <= 1e-12
        np.testing.assert_allclose(np.array(pa), np.array(pb), rtol=0, atol=1e-12)


@pytest.mark.parametrize("k", [3, 8, 11])
def test_ramp_variance_closed_form_box(k):
    # I1(i,j) = alpha*j: over a k x k box the values are uniform on alpha*{0..k-1}
    # (each once per row), so mu = alpha (j + (k-1)/2) and var = alpha^2 (k^2-1)/12.
    alpha = 3.0
    x = np.tile(alpha * np.arange(40, dtype=float), (25, 1))
    st = oracle.window_stats(x, x, oracle.box_window(k), 1)
    j = np.arange(st["mu1"].shape[1])
    np.testing.assert_allclose(st["mu1"], np.broadcast_to(alpha * (j + (k - 1) / 2), st["mu1"].shape),
                               rtol=1e-13)
    np.testing.assert_allclose(st["var1"], alpha ** 2 * (k * k - 1) / 12.0, rtol=1e-10)
    np.testing.assert_allclose(st["cov"], alpha ** 2 * (k * k - 1) / 12.0, rtol=1e-10)


def test_ramp_variance_closed_form_gaussian():
    # For a ramp along columns the 2-D variance is alpha^2 times the variance of
    # the 1-D Gaussian marginal (scipy's window, an independent route).
    k, sigma, alpha = 11, 1.5, 2.0
    x = np.tile(alpha * np.arange(30, dtype=float), (20, 1))
    st = oracle.window_stats(x, x, oracle.gaussian_window(k, sigma), 1)
    g = scipy.signal.windows.gaussian(k, std=sigma)
    g /= g.sum()
    t = np.arange(k)
    var = alpha ** 2 * (np.sum(g * t * t) - np.sum(g * t) ** 2)
    np.testing.assert_allclose(st["var1"], var, rtol=1e-9)


# --------------------------------------------------------------------------- SSIM formula

def _golden_rows():
    rows = []
    with open(GOLDEN) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append([float(t) for t in line.split()])
    return rows


@pytest.mark.parametrize("row", _golden_rows())
def test_constant_planes_closed_form(row):
    a, b, K1, K2, L, num, den = row
    x = np.full((16, 19), a)
    y = np.full((16, 19), b)
    for kind in ("gaussian", "box"):
        m, maps = oracle.ssim(x, y, kind, 11, 1.5, K1, K2, L)
        # fp64 rounding of sum w I^2 - mu^2 at I = 255 leaves ~1e-11 in cs
        np.testing.assert_allclose(maps["cs"], 1.0, rtol=0, atol=1e-10)
        np.testing.assert_allclose(maps["q"], num / den, rtol=1e-10)
        assert abs(m - num / den) < 1e-10
    # MS-SSIM of constant planes: l^beta_S (64 px survive 4 halvings to 4 px... use k=3)
    x = np.full((64, 64), a)
    y = np.full((64, 64), b)
    s, _ = oracle.msssim(x, y, scales=5, k=3, sigma=0.8, K1=K1, K2=K2, L=L)
    assert abs(s - (num / den) ** oracle.MSSSIM_EXPONENTS[-1]) < 1e-10


def test_mean_shift_gives_cs_one_and_luminance_closed_form():
    r = _rng(2)
    x = r.uniform(20, 200, (30, 31))
    c = 17.5
    m, maps = oracle.ssim(x, x + c)
    np.testing.assert_allclose(maps["cs"], 1.0, atol=1e-12)
    C1, _ = oracle.constants()
    mu = maps["mu1"]
    l = (2 * mu * (mu + c) + C1) / (mu ** 2 + (mu + c) ** 2 + C1)
    np.testing.assert_allclose(maps["l"], l, rtol=1e-12)
    np.testing.assert_allclose(maps["q"], l, rtol=1e-12)


def test_contrast_scaling_closed_form():
    # y = a x: cov = a var1, var2 = a^2 var1 => cs = (2 a v + C2)/((1+a^2) v + C2)
    r = _rng(3)
    x = r.uniform(0, 100, (25, 27))
    a = 0.6
    _, maps = oracle.ssim(x, a * x)
    _, C2 = oracle.constants()
    v = maps["var1"]
    np.testing.assert_allclose(maps["cs"], (2 * a * v + C2) / ((1 + a * a) * v + C2), rtol=1e-10)


def test_weber_rewrite_of_luminance():
    # Background section: mu2 = mu1 (1 + Lambda) gives
    # l = (2(1+Lambda) + C1/mu1^2) / (1 + (1+Lambda)^2 + C1/mu1^2).
    C1, _ = oracle.constants()
    for mu1, lam in [(50.0, 0.1), (200.0, -0.3), (10.0, 0.9)]:
        _, maps = oracle.ssim(np.full((12, 12), mu1), np.full((12, 12), mu1 * (1 + lam)))
        expect = (2 * (1 + lam) + C1 / mu1 ** 2) / (1 + (1 + lam) ** 2 + C1 / mu1 ** 2)
        np.testing.assert_allclose(maps["l"], expect, rtol=1e-12)


def test_identity_symmetry_boundedness():
    r = _rng(4)
    x = r.integers(0, 256, (40, 37)).astype(float)
    y = np.clip(x + r.normal(0, 30, x.shape), 0, 255)
    m, maps = oracle.ssim(x, x)
    assert m == 1.0 and np.all(maps["q"] == 1.0)          # unique maximum at I1 = I2
    m1, a = oracle.ssim(x, y)
    m2, b = oracle.ssim(y, x)
    np.testing.assert_allclose(a["q"], b["q"], rtol=0, atol=1e-13)  # symmetry (up to rounding order)
    assert abs(m1 - m2) < 1e-13 and m1 < 1.0
    neg = 255.0 - x                                         # anti-correlated patches
    for yy in (y, neg, np.zeros_like(x), np.full_like(x, 255.0)):
        _, mp = oracle.ssim(x, yy)
        assert np.all(np.abs(mp["q"]) <= 1.0 + 1e-15)      # boundedness
    _, mp = oracle.ssim(x, neg)
    assert mp["cs"].min() < 0                               # negative correlation occurs


@pytest.mark.parametrize("s", [2, 3, 4, 5])
def test_stride_is_subset_of_dense_map(s):
    r = _rng(5)
    x = r.uniform(0, 255, (41, 39))
    y = r.uniform(0, 255, (41, 39))
    _, d = oracle.ssim(x, y, stride=1)
    _, t = oracle.ssim(x, y, stride=s)
    np.testing.assert_array_equal(t["q"], d["q"][::s, ::s])
    assert t["q"].shape == ((41 - 11) // s + 1, (39 - 11) // s + 1)


# --------------------------------------------------------------------------- box / integral images

@pytest.mark.parametrize("shape,k,s", [((8, 8), 8, 1), ((33, 47), 8, 4), ((20, 25), 3, 1),
                                       ((50, 23), 11, 5), ((17, 17), 1, 2), ((40, 41), 7, 3)])
def test_integral_image_sums_equal_direct_sums_exactly(shape, k, s):
    r = _rng(6)
    x = r.integers(0, 256, shape).astype(np.uint8)
    y = r.integers(0, 256, shape).astype(np.uint8)
    a = oracle.box_sums(x, y, k, s, "integral")
    b = oracle.box_sums(x, y, k, s, "direct")
    np.testing.assert_array_equal(a, b)
    # numpy sliding windows: a third, independent route
    sw = lambda v: np.lib.stride_tricks.sliding_window_view(v.astype(np.int64), (k, k))[::s, ::s].sum(axis=(2, 3))
    xi, yi = x.astype(np.int64), y.astype(np.int64)
    for t, v in enumerate((xi, yi, xi * xi, yi * yi, xi * yi)):
        np.testing.assert_array_equal(a[..., t], sw(v))


def test_box_sums_extremes_fit_int64():
    x = np.full((16, 16), 255, np.uint8)
    a = oracle.box_sums(x, x, 16, 1)
    assert a[0, 0].tolist() == [255 * 256, 255 * 256, 65025 * 256, 65025 * 256, 65025 * 256]


@pytest.mark.parametrize("k,s", [(8, 4), (11, 1), (5, 2)])
def test_box_ssim_from_sums_equals_weighted_definition(k, s):
    r = _rng(7)
    x = r.integers(0, 256, (37, 45)).astype(np.uint8)
    y = np.clip(x.astype(int) + r.integers(-20, 21, x.shape), 0, 255).astype(np.uint8)
    m, q, cs, _ = oracle.box_ssim(x, y, k, s)
    m2, maps = oracle.ssim(x, y, "box", k, stride=s)
    np.testing.assert_allclose(q, maps["q"], atol=1e-12)
    np.testing.assert_allclose(cs, maps["cs"], atol=1e-12)
    assert abs(m - m2) < 1e-12


# --------------------------------------------------------------------------- MS-SSIM

@pytest.mark.parametrize("shape", [(10, 14), (11, 15), (1, 3), (7, 2)])
def test_downsample_is_2x2_mean_floor(shape):
    r = _rng(8)
    a = r.uniform(0, 255, shape)
    h, w = shape[0] // 2, shape[1] // 2
    ref = a[: 2 * h, : 2 * w].reshape(h, 2, w, 2).mean(axis=(1, 3))
    np.testing.assert_allclose(oracle.downsample2x2(a), ref, rtol=1e-15)


def test_downsample_exact_on_uint8_pyramid():
    # For uint8 input every scale-j value is an integer multiple of 4^-j: exact in fp32.
    r = _rng(9)
    a = r.integers(0, 256, (64, 96)).astype(float)
    for j in range(1, 5):
        a = oracle.downsample2x2(a)
        scaled = a * 4 ** j
        assert np.all(scaled == np.round(scaled))
        assert np.all(a.astype(np.float32).astype(np.float64) == a)
        assert scaled.min() >= 0 and scaled.max() <= 255 * 4 ** j <= 65535  # levels 1..4 fit 16 bits
    white = np.full((32, 32), 255.0)
    for _ in range(4):
        white = oracle.downsample2x2(white)
    assert np.all(white * 4 ** 4 == 65280)


def test_msssim_single_scale_is_ssim():
    r = _rng(10)
    x = r.uniform(0, 255, (30, 33))
    y = np.clip(x + r.normal(0, 10, x.shape), 0, 255)
    s, per = oracle.msssim(x, y, scales=1, exponents=(1.0,))
    m, _ = oracle.ssim(x, y)
    assert abs(s - m) < 1e-15 and abs(per[0][1] - m) < 1e-15


def test_msssim_identity_and_pyramid_recursion():
    r = _rng(11)
    x = r.uniform(0, 255, (180, 190))
    s, per = oracle.msssim(x, x)
    assert s == 1.0
    y = np.clip(x + r.normal(0, 12, x.shape), 0, 255)
    s, per = oracle.msssim(x, y)
    # scale 3 statistics must be those of the twice-downsampled pair
    x2 = x[:180, :188].reshape(45, 4, 47, 4).mean(axis=(1, 3))
    y2 = y[:180, :188].reshape(45, 4, 47, 4).mean(axis=(1, 3))
    m, maps = oracle.ssim(x2, y2)
    assert abs(per[2][0] - maps["cs"].mean()) < 1e-12
    exps = np.array(oracle.MSSSIM_EXPONENTS)
    mvec = np.array([p[0] for p in per[:-1]] + [per[-1][1]])
    assert abs(s - np.exp(np.sum(exps * np.log(mvec)))) < 1e-12
    ssum, _ = oracle.msssim(x, y, combine="sum")
    assert min(mvec) - 1e-15 <= ssum <= max(mvec) + 1e-15  # convex combination


def test_msssim_negative_pooled_cs_is_nan():
    r = _rng(12)
    x = r.uniform(0, 255, (96, 96))
    s, per = oracle.msssim(x, 255.0 - x, scales=3, exponents=(0.3, 0.3, 0.4), k=5, sigma=1.0)
    assert per[0][0] < 0 and math.isnan(s)


# --------------------------------------------------------------------------- gradient

def _fd(fun, y, h):
    g = np.empty_like(y)
    for idx in np.ndindex(y.shape):
        yp = y.copy(); yp[idx] += h
        ym = y.copy(); ym[idx] -= h
        g[idx] = (fun(yp) - fun(ym)) / (2 * h)
    return g


@pytest.mark.parametrize("kind,k,s,which,L", [("gaussian", 5, 1, "q", 255.0), ("gaussian", 5, 2, "cs", 255.0),
                                              ("box", 4, 1, "q", 1.0), ("gaussian", 11, 1, "q", 1.0)])
def test_gradient_matches_central_differences(kind, k, s, which, L):
    r = _rng(13)
    shape = (13, 14) if k < 11 else (14, 15)
    x = r.uniform(0, L, shape)
    y = x + r.normal(0, 0.1 * L, shape)
    g = oracle.ssim_grad(x, y, kind, k, 1.0, L=L, stride=s, which=which)

    def f(yy):
        _, maps = oracle.ssim(x, yy, kind, k, 1.0, L=L, stride=s)
        return maps[which].mean()

    fd = _fd(f, y, 1e-5 * L)
    np.testing.assert_allclose(g, fd, rtol=1e-6, atol=1e-9 * np.abs(fd).max())


def test_gradient_vanishes_at_identity():
    r = _rng(14)
    x = r.uniform(0, 255, (20, 22))
    g = oracle.ssim_grad(x, x)
    assert np.abs(g).max() < 1e-15


def test_gradient_sum_is_derivative_of_mean_shift_closed_form():
    # d/dc mean Q(x, x + c) = sum_q dQ/dy(q); with cs = 1 along the shift,
    # dl/dc = (2 mu B1 - 2 (mu + c) A1) / B1^2 from Eq. lum_term.
    r = _rng(15)
    x = r.uniform(30, 220, (24, 26))
    c = 5.0
    g = oracle.ssim_grad(x, x + c)
    _, maps = oracle.ssim(x, x + c)
    C1, _ = oracle.constants()
    mu = maps["mu1"]
    A1 = 2 * mu * (mu + c) + C1
    B1 = mu ** 2 + (mu + c) ** 2 + C1
    dldc = (2 * mu * B1 - 2 * (mu + c) * A1) / B1 ** 2
    assert abs(g.sum() - dldc.mean()) < 1e-12 * max(1.0, abs(dldc.mean())) + 1e-15


def test_msssim_gradient_matches_central_differences():
    r = _rng(16)
    x = r.uniform(0, 255, (26, 28))
    y = np.clip(x + r.normal(0, 20, x.shape), 0, 255)
    kw = dict(scales=3, exponents=(0.3, 0.3, 0.4), k=3, sigma=0.8)
    _, g = oracle.msssim_grad(x, y, **kw)
    fd = _fd(lambda yy: oracle.msssim(x, yy, **kw)[0], y, 1e-3)
    # central differences carry ~eps*f/h = 1e-13 of rounding noise here
    np.testing.assert_allclose(g, fd, rtol=1e-5, atol=1e-6 * np.abs(fd).max())
    _, gs = oracle.msssim_grad(x, y, combine="sum", **kw)
    fds = _fd(lambda yy: oracle.msssim(x, yy, combine="sum", **kw)[0], y, 1e-3)
    np.testing.assert_allclose(gs, fds, rtol=1e-5, atol=1e-6 * np.abs(fds).max())


# --------------------------------------------------------------------------- colour / temporal

def test_colour_combination():
    assert oracle.colour_score(0.9, 0.9, 0.9) == pytest.approx(0.9, abs=1e-15)
    assert oracle.colour_score(0.8, 0.4, 0.0) == pytest.approx((6 * 0.8 + 0.4) / 8, abs=1e-15)
    # FFMPEG / Daala weights 0.8 / 0.1 / 0.1 (Section "Channel-wise SSIM")
    assert oracle.colour_score(1.0, 0.5, 0.0, (0.8, 0.1, 0.1)) == pytest.approx(0.85, abs=1e-15)
    # alpha = beta = -0.3 (the paper's optimum): F = (f_Y - 0.3 f_Cb - 0.3 f_Cr)/0.4
    assert oracle.colour_score(0.9, 0.5, 0.7, (1.0, -0.3, -0.3)) == pytest.approx((0.9 - 0.15 - 0.21) / 0.4)


def test_temporal_pooling():
    v = np.array([0.9, 0.5, 0.7, 0.95, 0.6, 0.8, 0.85, 0.75, 0.65, 0.99, 0.55])
    m, p10, pp = oracle.temporal_pool(v, 10.0, r=4.0)
    assert m == pytest.approx(v.mean(), abs=1e-15)
    assert p10 == pytest.approx(np.percentile(v, 10.0), abs=1e-15)   # library routine
    # n = 11: h = 1.0 -> the second smallest value exactly; PP divides {0.5, 0.55} by r
    assert p10 == 0.55
    assert pp == pytest.approx((v.sum() - 0.5 - 0.55 + (0.5 + 0.55) / 4.0) / 11, abs=1e-15)
    # r = 1 leaves every score unchanged: PP reduces to the mean (Section "Percentile Pooling")
    assert oracle.temporal_pool(v, 10.0, r=1.0)[2] == pytest.approx(m, abs=1e-15)
    r = _rng(17)
    w = r.uniform(0.5, 1.0, 120)
    _, p, _ = oracle.temporal_pool(w, 10.0)
    assert p == pytest.approx(np.percentile(w, 10.0), abs=1e-15)


# ------------------------------------------------------------------ border extension

def _embed_zero(a, before, after):
    """Zero extension built by slice assignment (independent of np.pad)."""
    H, W = a.shape
    out = np.zeros((H + before + after, W + before + after))
    out[before:before + H, before:before + W] = a
    return out


def _mirror_index(n, before, after):
    """Indices of the half-sample mirror extension, x(-1-i) = x(i), x(n+i) = x(n-1-i)."""
    left = list(range(before - 1, -1, -1))
    right = list(range(n - 1, n - 1 - after, -1))
    return np.array(left + list(range(n)) + right)


@pytest.mark.parametrize("k", [11, 8, 3])
def test_border_extension_layout(k):
    r = np.random.default_rng(40)
    a = r.uniform(0, 255, (23, 31))
    before, after = (k - 1) // 2, k - 1 - (k - 1) // 2
    np.testing.assert_array_equal(oracle.extend_border(a, k, "zero"), _embed_zero(a, before, after))
    ri, ci = _mirror_index(23, before, after), _mirror_index(31, before, after)
    np.testing.assert_array_equal(oracle.extend_border(a, k, "reflect"), a[np.ix_(ri, ci)])
    np.testing.assert_array_equal(oracle.extend_border(a, k, "valid"), a)


@pytest.mark.parametrize("border", ["zero", "reflect"])
def test_border_maps_have_one_output_per_pixel_and_keep_the_interior(border):
    r = np.random.default_rng(41)
    x = r.uniform(0, 255, (40, 52))
    y = np.clip(x + r.normal(0, 9, x.shape), 0, 255)
    _, valid = oracle.ssim(x, y)
    _, ext = oracle.ssim(x, y, border=border)
    assert ext["q"].shape == x.shape
    # windows wholly inside the image are the valid map, shifted by the border
    np.testing.assert_allclose(ext["q"][5:-5, 5:-5], valid["q"], rtol=0, atol=1e-13)
    # stride: the strided extended map keeps every s-th output
    _, ext2 = oracle.ssim(x, y, border=border, stride=3)
    np.testing.assert_allclose(ext2["q"], ext["q"][::3, ::3], rtol=0, atol=1e-13)


def test_reflect_border_of_a_constant_image_is_constant():
    x = np.full((30, 30), 90.0)
    y = np.full((30, 30), 120.0)
    C1, _ = oracle.constants()
    _, m = oracle.ssim(x, y, border="reflect")
    np.testing.assert_allclose(m["q"], (2 * 90 * 120 + C1) / (90 ** 2 + 120 ** 2 + C1), rtol=1e-10)
    # zero extension lowers the corner means: the corner window sees 36 of 121 pixels weighted
    _, z = oracle.ssim(x, y, border="zero", window_kind="box")
    f = 36 / 121
    mx, my = 90 * f, 120 * f
    vx, vy, cxy = 90 ** 2 * f - mx ** 2, 120 ** 2 * f - my ** 2, 90 * 120 * f - mx * my
    _, C2 = oracle.constants()
    q00 = (2 * mx * my + C1) / (mx ** 2 + my ** 2 + C1) * (2 * cxy + C2) / (vx + vy + C2)
    assert z["q"][0, 0] == pytest.approx(q00, rel=1e-12)


def test_msssim_border_uses_unextended_pyramid():
    r = np.random.default_rng(42)
    x = r.uniform(0, 255, (96, 112))
    y = np.clip(x + r.normal(0, 12, x.shape), 0, 255)
    s, per = oracle.msssim(x, y, scales=3, exponents=(0.3, 0.3, 0.4), border="zero")
    a, b = x, y
    for j in range(3):
        _, m = oracle.ssim(a, b, border="zero")
        assert per[j][0] == pytest.approx(m["cs"].mean(), abs=1e-14)
        assert per[j][1] == pytest.approx(m["q"].mean(), abs=1e-14)
        a, b = oracle.downsample2x2(a), oracle.downsample2x2(b)
