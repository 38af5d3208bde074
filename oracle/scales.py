"""FP64 oracle of the scale handling around SSIM / MS-SSIM (Section
"Salient Features of SSIM and MS-SSIM Implementations" and Section
"Transforming across Various Scales" of arXiv 2101.06354): the automatic
downscaling factor and block-mean downscaling, and the 9/7 biorthogonal
wavelet low-pass used as the MS-SSIM pyramid by one implementation.

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle``.  Pinned by
``tests/test_oracle_scales.py``.
"""
from __future__ import annotations

import math

import numpy as np

#: Low-pass analysis filter of the Cohen-Daubechies-Feauveau 9/7 wavelet
#: (the JPEG 2000 irreversible transform), scaled to sum to one, taps -4..4.
CDF97_LOWPASS = np.array([0.026748757410810, -0.016864118442875, -0.078223266528990, 0.266864118442875,
                          0.602949018236360, 0.266864118442875, -0.078223266528990, -0.016864118442875,
                          0.026748757410810])
CDF97_LOWPASS = CDF97_LOWPASS / CDF97_LOWPASS.sum()


def downscale_factor(h: int, w: int, rule: str = "round_min") -> int:
    """Automatic downscaling factor Z.  rule "round_min": max(1, round(min(H,
    W)/256)) (the recommended implementation and LIBVMAF: the smaller side
    brought to about 256); rule "ceil_h": max(1, ceil(H/256)) (the transform
    the paper quotes for scale-based models).  Reading: round() rounds halves
    up, as the integer division (n + 128) / 256 does."""
    if rule == "round_min":
        return max(1, (min(h, w) + 128) // 256)
    if rule == "ceil_h":
        return max(1, math.ceil(h / 256))
    raise ValueError(rule)


def downscale_block(img, z: int) -> np.ndarray:
    """Z x Z block mean with floor size (H // Z, W // Z): the averaging filter
    of width Z followed by keeping every Z-th sample.  Reading: the blocks do
    not overlap, like the 2x2 MS-SSIM pyramid (Z = 2 gives it exactly)."""
    a = np.asarray(img, dtype=np.float64)
    h, w = a.shape[0] // z, a.shape[1] // z
    out = np.zeros((h, w))
    for m in range(z):
        for n in range(z):
            out += a[m:m + z * h:z, n:n + z * w:z]
    return out / (z * z)


def _sym(i: int, n: int) -> int:
    """Whole-sample symmetric extension index (... 2 1 | 0 1 2 ... n-1 | n-2 ...)."""
    if n == 1:
        return 0
    period = 2 * (n - 1)
    i = i % period
    return i if i < n else period - i


def pyramid_97(img) -> np.ndarray:
    """One dyadic step of the 9/7 wavelet pyramid: the CDF 9/7 low-pass
    analysis filter applied along rows and columns with whole-sample
    symmetric extension, keeping the even samples.  Reading: output size
    floor(H/2) x floor(W/2) like the 2x2 average pyramid; output (i, j) is
    centred on input (2i, 2j)."""
    a = np.asarray(img, dtype=np.float64)
    H, W = a.shape
    h, w = H // 2, W // 2
    rows = np.zeros((H, w))
    for j in range(w):
        for t in range(-4, 5):
            rows[:, j] += CDF97_LOWPASS[t + 4] * a[:, _sym(2 * j + t, W)]
    out = np.zeros((h, w))
    for i in range(h):
        for t in range(-4, 5):
            out[i, :] += CDF97_LOWPASS[t + 4] * rows[_sym(2 * i + t, H), :]
    return out


def rgb_to_ycbcr(r, g, b):
    """BT.709 luma and colour differences as the paper prints them (Section
    "Channel-wise SSIM"): Y = 0.213 R + 0.715 G + 0.072 B, Cb = 0.539 (B - Y),
    Cr = 0.635 (R - Y), on the planes' own scale (no offset, no clipping)."""
    r, g, b = (np.asarray(t, dtype=np.float64) for t in (r, g, b))
    y = 0.213 * r + 0.715 * g + 0.072 * b
    return y, 0.539 * (b - y), 0.635 * (r - y)
