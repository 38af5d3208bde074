"""FP64 CPU oracle for SSIM / MS-SSIM (arXiv 2101.06354).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The CUDA library never calls it and shares no code with it.

The window statistics, SSIM terms, integral images, downsampling and the
gradient are plain C (``ssim_oracle.c``); this module marshals numpy arrays
into it and writes the multi-scale, colour and temporal combinations out in
numpy, each function citing the passage of the paper it follows.

Parity status: every function here is pinned by ``tests/test_oracle_pins.py``
(closed forms, invariants, library routines on small inputs, finite
differences); none is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np

from .build import build_oracle

_lib = None

#: MS-SSIM scale exponents used by the paper's MS-SSIM implementations
#: (Introduction: five dyadic scales combined by exponential weighting).  The
#: paper does not print them; these are the values of the original MS-SSIM.
MSSSIM_EXPONENTS = (0.0448, 0.2856, 0.3001, 0.2363, 0.1333)

_dp = ctypes.POINTER(ctypes.c_double)
_i64p = ctypes.POINTER(ctypes.c_int64)
_u8p = ctypes.POINTER(ctypes.c_uint8)


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build_oracle())
        L, I = ctypes.c_long, ctypes.c_int
        D = ctypes.c_double
        lib.oracle_gaussian_window.argtypes = [I, D, _dp]
        lib.oracle_box_window.argtypes = [I, _dp]
        lib.oracle_window_stats.argtypes = [_dp, _dp, L, L, _dp, I, I, _dp, _dp, _dp, _dp, _dp]
        lib.oracle_ssim_terms.argtypes = [_dp, _dp, _dp, _dp, _dp, L, D, D, _dp, _dp, _dp]
        lib.oracle_mean.argtypes = [_dp, L]
        lib.oracle_mean.restype = D
        lib.oracle_box_sums_direct.argtypes = [_u8p, _u8p, L, L, L, I, I, _i64p]
        lib.oracle_box_sums_integral.argtypes = [_u8p, _u8p, L, L, L, I, I, _i64p]
        lib.oracle_box_ssim_from_sums.argtypes = [_i64p, L, I, D, D, _dp, _dp]
        lib.oracle_box3d_sums_direct.argtypes = [_u8p, _u8p, L, L, L, L, L, I, I, _i64p]
        lib.oracle_box_ssim_from_sums_n.argtypes = [_i64p, L, D, D, D, _dp, _dp]
        lib.oracle_downsample2x2.argtypes = [_dp, L, L, _dp]
        lib.oracle_ssim_grad.argtypes = [_dp, _dp, L, L, _dp, I, I, D, D, I, _dp]
        lib.oracle_num_threads.restype = I
        lib.oracle_set_num_threads.argtypes = [I]
        lib.oracle_set_num_threads.restype = None
        lib.oracle_window_stats_separable.argtypes = [_dp, _dp, L, L, _dp, I, I, _dp, _dp, _dp, _dp, _dp]
        _lib = lib
    return _lib


def _ptr(a, t=_dp):
    return a.ctypes.data_as(t)


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _check(rc):
    if rc != 0:
        raise ValueError("oracle rejected its arguments (rc=%d)" % rc)


def num_threads() -> int:
    """Threads the oracle's OpenMP split uses."""
    return int(_load().oracle_num_threads())


def set_num_threads(n: int) -> None:
    """Threads of the OpenMP split from now on (the CPU baseline times one
    core and all cores)."""
    _load().oracle_set_num_threads(int(n))


def out_shape(h: int, w: int, k: int, stride: int):
    """Valid, strided map size (Section "Effect of stride"): floor((n-k)/s)+1."""
    return ((h - k) // stride + 1, (w - k) // stride + 1)


def constants(K1: float = 0.01, K2: float = 0.03, L: float = 255.0):
    """C1 = (K1 L)^2, C2 = (K2 L)^2 (Background section)."""
    return (K1 * L) ** 2, (K2 * L) ** 2


def gaussian_window(k: int = 11, sigma: float = 1.5) -> np.ndarray:
    """k x k Gaussian weights summing to one (Background section)."""
    w = np.empty((k, k), np.float64)
    _check(_load().oracle_gaussian_window(k, sigma, _ptr(w)))
    return w


def box_window(k: int) -> np.ndarray:
    """k x k rectangular weights 1/k^2."""
    w = np.empty((k, k), np.float64)
    _check(_load().oracle_box_window(k, _ptr(w)))
    return w


def taps_1d(kind: str, k: int, sigma: float = 1.5) -> np.ndarray:
    """1-D factor g of a separable window w = g g^T: the Gaussian
    exp(-(t-c)^2 / 2 sigma^2) normalised to sum 1, or the box 1/k."""
    if kind == "gaussian":
        c = 0.5 * (k - 1)
        t = np.arange(k, dtype=np.float64)
        v = np.exp(-((t - c) ** 2) / (2.0 * sigma * sigma))
        return v / v.sum()
    if kind == "box":
        return np.full(k, 1.0 / k)
    raise ValueError(kind)


def window(kind: str, k: int, sigma: float = 1.5) -> np.ndarray:
    if kind == "gaussian":
        return gaussian_window(k, sigma)
    if kind == "box":
        return box_window(k)
    raise ValueError(kind)


def gaussian_k_for_sigma(sigma: float) -> int:
    """Window width for a Gaussian of scale sigma.

    Section "Effect of window size" truncates at about 7 sigma and forces an
    odd width; this helper takes 2*floor(3.5 sigma)+1 (11 at sigma = 1.5,
    the same as MATLAB's 2*ceil(3 sigma)+1 there).
    """
    return 2 * int(math.floor(3.5 * sigma)) + 1


def rect_k_equivalent(sigma: float, rule: str = "variance") -> int:
    """Rectangular window size 2K+1 matched to a Gaussian (Section "Effect of
    window size"): same variance K = ceil(sigma sqrt 3); same 3 dB bandwidth
    K = ceil(1.602 sigma)."""
    if rule == "variance":
        K = math.ceil(sigma * math.sqrt(3.0))
    elif rule == "bandwidth":
        K = math.ceil(1.602 * sigma)
    else:
        raise ValueError(rule)
    return 2 * K + 1


def window_stats(x, y, w, stride: int = 1):
    """Eqs. local_means .. local_corr at every valid strided position."""
    x, y, w = _f64(x), _f64(y), _f64(w)
    H, W = x.shape
    k = w.shape[0]
    if y.shape != x.shape or w.shape != (k, k) or H < k or W < k or stride < 1:
        raise ValueError("bad shapes")
    oh, ow = out_shape(H, W, k, stride)
    maps = [np.empty((oh, ow), np.float64) for _ in range(5)]
    _check(_load().oracle_window_stats(_ptr(x), _ptr(y), H, W, _ptr(w), k, stride,
                                       *[_ptr(m) for m in maps]))
    return dict(zip(("mu1", "mu2", "var1", "var2", "cov"), maps))


def window_stats_separable(x, y, g, stride: int = 1):
    """The statistics of window_stats for the separable window g g^T, by a
    row pass then a column pass (the mode the CPU baseline times)."""
    x, y, g = _f64(x), _f64(y), _f64(g)
    H, W = x.shape
    k = g.shape[0]
    if y.shape != x.shape or g.ndim != 1 or H < k or W < k or stride < 1:
        raise ValueError("bad shapes")
    oh, ow = out_shape(H, W, k, stride)
    maps = [np.empty((oh, ow), np.float64) for _ in range(5)]
    _check(_load().oracle_window_stats_separable(_ptr(x), _ptr(y), H, W, _ptr(g), k, stride,
                                                 *[_ptr(m) for m in maps]))
    return dict(zip(("mu1", "mu2", "var1", "var2", "cov"), maps))


def ssim_terms(st, C1: float, C2: float):
    """Eq. lum_term and the C3 = C2/2 contrast-structure term; returns l, cs, Q."""
    n = st["mu1"].size
    l, cs, q = (np.empty(st["mu1"].shape, np.float64) for _ in range(3))
    _check(_load().oracle_ssim_terms(*[_ptr(st[k]) for k in ("mu1", "mu2", "var1", "var2", "cov")],
                                     n, C1, C2, _ptr(l), _ptr(cs), _ptr(q)))
    return l, cs, q


def mean(v) -> float:
    """Mean pooling over the map elements that exist (Background section)."""
    v = _f64(v).ravel()
    return float(_load().oracle_mean(_ptr(v), v.size))


def extend_border(img, k: int, border: str = "valid") -> np.ndarray:
    """The image extended for a k x k window (Section "Salient Features of
    SSIM and MS-SSIM Implementations", the border-handling column: zero
    padding, reflection padding, or only valid outputs).  Reading:
    floor((k-1)/2) rows / columns before and the rest of k-1 after, so the
    valid windows of the extended image give one output per input pixel at
    stride 1; "zero" fills with 0, "reflect" mirrors about the image border
    with the edge sample repeated (x(-1-i) = x(i), x(H+i) = x(H-1-i));
    "valid" returns the image unchanged."""
    a = _f64(img)
    if border == "valid":
        return a
    before = (k - 1) // 2
    after = k - 1 - before
    H, W = a.shape
    if border == "zero":
        return np.pad(a, ((before, after), (before, after)), mode="constant")
    if border == "reflect":
        if min(H, W) < after:
            raise ValueError("image smaller than the mirrored border")
        return np.pad(a, ((before, after), (before, after)), mode="symmetric")
    raise ValueError(border)


def ssim(x, y, window_kind: str = "gaussian", k: int = 11, sigma: float = 1.5,
         K1: float = 0.01, K2: float = 0.03, L: float = 255.0, stride: int = 1, border: str = "valid"):
    """SSIM map and MSSIM of one pair; border = "valid" (only windows inside
    the image), "zero" or "reflect" (extend_border first).

    Returns ``(mssim, maps)`` with maps = {"q", "cs", "l", and the statistics}.
    """
    C1, C2 = constants(K1, K2, L)
    x, y = extend_border(x, k, border), extend_border(y, k, border)
    st = window_stats(x, y, window(window_kind, k, sigma), stride)
    l, cs, q = ssim_terms(st, C1, C2)
    maps = dict(st, l=l, cs=cs, q=q)
    return mean(q), maps


def box_sums(x, y, k: int, stride: int = 1, method: str = "integral"):
    """Exact int64 window sums (S1_1, S1_2, S2_1, S2_2, S12) of a uint8 pair,
    shape (OH, OW, 5).  method="integral" follows the paper's summed-area-table
    algorithm (Eqs. integral_image_start .. integral_image_end);
    method="direct" sums each window."""
    x = np.ascontiguousarray(x, dtype=np.uint8)
    y = np.ascontiguousarray(y, dtype=np.uint8)
    H, W = x.shape
    if y.shape != x.shape or H < k or W < k or stride < 1 or k < 1:
        raise ValueError("bad shapes")
    oh, ow = out_shape(H, W, k, stride)
    out = np.empty((oh, ow, 5), np.int64)
    fn = {"integral": _load().oracle_box_sums_integral,
          "direct": _load().oracle_box_sums_direct}[method]
    _check(fn(_ptr(x, _u8p), _ptr(y, _u8p), H, W, W, k, stride, _ptr(out, _i64p)))
    return out


def box_ssim(x, y, k: int = 8, stride: int = 4, K1: float = 0.01, K2: float = 0.03,
             L: float = 255.0):
    """Rectangular-window SSIM of a uint8 pair through integral images
    (Eqs. mean_from_sum .. corr_from_sum).  Returns (mssim, q_map, cs_map, sums)."""
    C1, C2 = constants(K1, K2, L)
    sums = box_sums(x, y, k, stride, "integral")
    n = sums.shape[0] * sums.shape[1]
    q = np.empty(sums.shape[:2], np.float64)
    cs = np.empty(sums.shape[:2], np.float64)
    _check(_load().oracle_box_ssim_from_sums(_ptr(sums, _i64p), n, k, C1, C2, _ptr(q), _ptr(cs)))
    return mean(q), q, cs, sums


def box3d_sums(x, y, k: int = 11, kt: int = 5) -> np.ndarray:
    """SSIM-3D window sums (Section "Spatio-Temporal SSIM"): the five exact
    int64 sums of every k x k x kt neighbourhood of a uint8 video pair
    (T, H, W), shape (T-kt+1, H-k+1, W-k+1, 5); output frame t covers input
    frames t .. t+kt-1 (the window ending at frame t+kt-1)."""
    x = np.ascontiguousarray(x, dtype=np.uint8)
    y = np.ascontiguousarray(y, dtype=np.uint8)
    T, H, W = x.shape
    if y.shape != x.shape or T < kt or H < k or W < k or k < 1 or kt < 1:
        raise ValueError("bad shapes")
    out = np.empty((T - kt + 1, H - k + 1, W - k + 1, 5), np.int64)
    _check(_load().oracle_box3d_sums_direct(_ptr(x, _u8p), _ptr(y, _u8p), T, H, W, W, H * W, k, kt,
                                            _ptr(out, _i64p)))
    return out


def ssim3d(x, y, k: int = 11, kt: int = 5, K1: float = 0.01, K2: float = 0.03, L: float = 255.0):
    """SSIM-3D of a uint8 video pair (T, H, W) (Section "Spatio-Temporal
    SSIM"): SSIM whose local statistics are taken over k x k x kt rectangular
    spatio-temporal neighbourhoods.  Reading: like the spatial map, only
    windows inside the video count, so output frames are the T-kt+1 frames
    with a full temporal window.  Returns (video score, per-frame mean Q of
    the T-kt+1 output frames, Q maps)."""
    C1, C2 = constants(K1, K2, L)
    sums = box3d_sums(x, y, k, kt)
    n = sums.shape[0] * sums.shape[1] * sums.shape[2]
    q = np.empty(sums.shape[:3], np.float64)
    _check(_load().oracle_box_ssim_from_sums_n(_ptr(sums, _i64p), n, float(k * k * kt), C1, C2, _ptr(q), None))
    frames = np.array([mean(q[t]) for t in range(q.shape[0])])
    return float(frames.sum() / frames.size), frames, q


def _box3d_stats(x, y, k: int, kt: int):
    """Means, variances and covariance over every k x k x kt neighbourhood of
    a float video pair (T, H, W), by direct fp64 summation of the window."""
    a, b = _f64(x), _f64(y)
    T, H, W = a.shape
    ot, oh, ow = T - kt + 1, H - k + 1, W - k + 1
    s = [np.zeros((ot, oh, ow)) for _ in range(5)]
    for o in range(kt):
        for m in range(k):
            for n in range(k):
                pa, pb = a[o:o + ot, m:m + oh, n:n + ow], b[o:o + ot, m:m + oh, n:n + ow]
                s[0] += pa
                s[1] += pb
                s[2] += pa * pa
                s[3] += pb * pb
                s[4] += pa * pb
    N = float(k * k * kt)
    mu1, mu2 = s[0] / N, s[1] / N
    return mu1, mu2, s[2] / N - mu1 * mu1, s[3] / N - mu2 * mu2, s[4] / N - mu1 * mu2


def msssim3d(x, y, k: int = 11, kt: int = 5, scales: int = 5, exponents=MSSSIM_EXPONENTS,
             combine: str = "product", K1: float = 0.01, K2: float = 0.03, L: float = 255.0):
    """MS-SSIM-3D (Section "Spatio-Temporal SSIM": 3-D SSIM computed over
    multiple spatial scales) of a video pair (T, H, W).  Reading: each frame
    has its own 2x2 average pyramid; at every level the k x k x kt box
    statistics give cs and Q maps for the T-kt+1 output frames; per output
    frame, m_j = mean cs_j (j < S) and m_S = mean Q_S are combined as in
    MS-SSIM; the video score is the temporal mean.  Returns (video score,
    per-frame scores, per-level (T-kt+1, 2) of (mean cs_j, mean Q_j))."""
    exps = np.asarray(exponents[:scales], np.float64)
    C1, C2 = constants(K1, K2, L)
    a, b = _f64(x), _f64(y)
    per = []
    for j in range(scales):
        mu1, mu2, v1, v2, cv = _box3d_stats(a, b, k, kt)
        lum = (2 * mu1 * mu2 + C1) / (mu1 * mu1 + mu2 * mu2 + C1)
        cs = (2 * cv + C2) / (v1 + v2 + C2)
        per.append(np.stack([cs.mean(axis=(1, 2)), (lum * cs).mean(axis=(1, 2))], axis=1))
        if j + 1 < scales:
            a = np.stack([downsample2x2(f) for f in a])
            b = np.stack([downsample2x2(f) for f in b])
    m = np.stack([per[j][:, 0] for j in range(scales - 1)] + [per[-1][:, 1]], axis=1)
    if combine == "product":
        with np.errstate(invalid="ignore"):
            frames = np.prod(np.power(m, exps), axis=1)
    else:
        frames = (m * (exps / exps.sum())).sum(axis=1)
    return float(frames.sum() / frames.size), frames, per


def downsample2x2(img) -> np.ndarray:
    """2x2 average pooling, floor size (Daala / Scikit-Video / Tensorflow MS-SSIM)."""
    img = _f64(img)
    H, W = img.shape
    out = np.empty((H // 2, W // 2), np.float64)
    _check(_load().oracle_downsample2x2(_ptr(img), H, W, _ptr(out)))
    return out


def msssim(x, y, scales: int = 5, exponents=MSSSIM_EXPONENTS, combine: str = "product",
           window_kind: str = "gaussian", k: int = 11, sigma: float = 1.5,
           K1: float = 0.01, K2: float = 0.03, L: float = 255.0, pyramid: str = "avg2",
           border: str = "valid", mode: str = "direct"):
    """MS-SSIM (Introduction; Section "Salient Features ...").

    Scale 1 is the input; scale j+1 is the 2x2 average of scale j
    (pyramid="avg2"), or its 9/7 wavelet low-pass (pyramid="97",
    ``oracle.scales.pyramid_97``, the LIBVMAF variant of that section).  The
    contrast-structure term is pooled at every scale and the luminance term
    only at the coarsest: m_j = mean cs_j for j < S and m_S = mean Q_S.
    combine="product": prod_j m_j^beta_j.  combine="sum" (Scikit-Video):
    sum_j (beta_j / sum beta) m_j, a convex combination.  With border "zero"
    or "reflect" each level is extended (extend_border) for its own SSIM
    map; the pyramid is formed from the unextended levels.
    mode="direct" (the checker) sums every k x k window; mode="separable"
    takes the row-then-column passes of window_stats_separable (equal to
    rounding; the CPU baseline's mode).
    Returns (score, per_scale) with per_scale[j] = (mean cs_j, mean Q_j).
    """
    exps = np.asarray(exponents[:scales], np.float64)
    if len(exps) != scales:
        raise ValueError("need one exponent per scale")
    C1, C2 = constants(K1, K2, L)
    if mode == "direct":
        w = window(window_kind, k, sigma)
        stats = window_stats
    elif mode == "separable":
        w = taps_1d(window_kind, k, sigma)
        stats = window_stats_separable
    else:
        raise ValueError(mode)
    a, b = _f64(x), _f64(y)
    per = []
    for j in range(scales):
        st = stats(extend_border(a, k, border), extend_border(b, k, border), w, 1)
        _, cs, q = ssim_terms(st, C1, C2)
        per.append((mean(cs), mean(q)))
        if j + 1 < scales:
            if pyramid == "avg2":
                a, b = downsample2x2(a), downsample2x2(b)
            elif pyramid == "97":
                from .scales import pyramid_97

                a, b = pyramid_97(a), pyramid_97(b)
            else:
                raise ValueError(pyramid)
    m = np.array([per[j][0] for j in range(scales - 1)] + [per[-1][1]])
    if combine == "product":
        with np.errstate(invalid="ignore"):
            score = float(np.prod(np.power(m, exps)))
    elif combine == "sum":
        score = float(np.sum(exps / exps.sum() * m))
    else:
        raise ValueError(combine)
    return score, per


def ssim_grad(x, y, window_kind: str = "gaussian", k: int = 11, sigma: float = 1.5,
              K1: float = 0.01, K2: float = 0.03, L: float = 255.0, stride: int = 1,
              which: str = "q") -> np.ndarray:
    """d(mean Q)/dy (which="q") or d(mean cs)/dy (which="cs"); chain rule of
    the Background-section definition (see ssim_oracle.c)."""
    C1, C2 = constants(K1, K2, L)
    x, y = _f64(x), _f64(y)
    w = window(window_kind, k, sigma)
    g = np.empty_like(y)
    H, W = y.shape
    _check(_load().oracle_ssim_grad(_ptr(x), _ptr(y), H, W, _ptr(w), k, stride, C1, C2,
                                    {"q": 0, "cs": 1}[which], _ptr(g)))
    return g


def msssim_grad(x, y, scales: int = 5, exponents=MSSSIM_EXPONENTS, combine: str = "product",
                window_kind: str = "gaussian", k: int = 11, sigma: float = 1.5,
                K1: float = 0.01, K2: float = 0.03, L: float = 255.0):
    """d(MS-SSIM)/dy by the chain rule through the scale combination and the
    2x2 average pooling (its adjoint spreads a quarter of each coarse gradient
    to the four pixels it averaged)."""
    score, per = msssim(x, y, scales, exponents, combine, window_kind, k, sigma, K1, K2, L)
    exps = np.asarray(exponents[:scales], np.float64)
    m = np.array([per[j][0] for j in range(scales - 1)] + [per[-1][1]])
    if combine == "product":
        dscore_dm = score * exps / m
    else:
        dscore_dm = exps / exps.sum()
    xs, ys = [_f64(x)], [_f64(y)]
    for _ in range(scales - 1):
        xs.append(downsample2x2(xs[-1]))
        ys.append(downsample2x2(ys[-1]))
    g = None
    for j in reversed(range(scales)):
        gj = dscore_dm[j] * ssim_grad(xs[j], ys[j], window_kind, k, sigma, K1, K2, L, 1,
                                      "q" if j == scales - 1 else "cs")
        if g is not None:
            up = np.zeros_like(gj)
            h2, w2 = g.shape
            up[: 2 * h2, : 2 * w2] = 0.25 * np.repeat(np.repeat(g, 2, 0), 2, 1)
            gj = gj + up
        g = gj
    return score, g


def colour_score(s_y: float, s_u: float, s_v: float, weights=(6.0, 1.0, 1.0)) -> float:
    """Channel-weighted colour SSIM (Section "Channel-wise SSIM"):
    F = (f_Y + alpha f_Cb + beta f_Cr) / (1 + alpha + beta); weights are
    (w_Y, w_U, w_V) = (1, alpha, beta) up to scale, e.g. 6:1:1 or 0.8/0.1/0.1."""
    wy, wu, wv = (float(t) for t in weights)
    return (wy * s_y + wu * s_u + wv * s_v) / (wy + wu + wv)


def temporal_pool(frame_scores, percentile: float = 10.0, r: float = 4.0):
    """Temporal pooling of frame scores (Section "Spatio-temporal Aggregation
    of Quality Scores"): the temporal mean; the p-th percentile of the scores
    by linear interpolation between order statistics (position
    h = p/100 (n-1) in the sorted list); and percentile pooling (Section
    "Percentile Pooling"): every score in the lowest p percent (at or below
    that percentile) is divided by r and the results are averaged,
    S_PP = (1/n) sum_t Q~(t) with Q~ = Q/r in the lowest p percent, else Q."""
    v = np.sort(_f64(frame_scores).ravel())
    n = v.size
    mean_ = float(v.sum() / n)
    h = percentile / 100.0 * (n - 1)
    lo = int(math.floor(h))
    hi = min(lo + 1, n - 1)
    pct = float(v[lo] + (h - lo) * (v[hi] - v[lo]))
    w = np.where(v <= pct, v / r, v)
    return mean_, pct, float(w.sum() / n)
