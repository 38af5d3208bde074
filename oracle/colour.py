"""FP64 oracle of CMSSIM (Section "CMSSIM" of arXiv 2101.06354): SSIM of the
CIELAB lightness weighted by the colour difference of the chromatically
smoothed images.

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle``.  Pinned by
``tests/test_oracle_colour.py``.

The steps follow the section in its order: linear RGB -> CIE XYZ -> the
luminance / red-green / blue-yellow planes (Q1, Q2, Q3; the paper's forward
matrix) -> Gaussian smoothing of the two chromatic planes -> back to XYZ (the
paper's inverse matrix, as printed) -> CIELAB -> Delta E per pixel; the SSIM
map weighted by (1 - Delta E / 45) and mean-pooled.  Readings of what the
section leaves open:
  * input: linear RGB in [0, 1] (uint8 divided by 255), no transfer curve;
    RGB -> XYZ with the BT.709 / sRGB primaries and D65 white (IEC 61966-2-1);
  * the smoothing kernel: the SSIM Gaussian window (k taps, sigma), one
    output per pixel, the planes extended by mirroring about the border;
  * CIELAB: the CIE 1976 definition relative to the D65 white of the same
    matrix, with the linear segment below (6/29)^3;
  * the SSIM map: the Background-section SSIM of the L* planes (dynamic range
    L = 100) with valid windows; each map value is weighted by Delta E at its
    window's centre pixel.
"""
from __future__ import annotations

import numpy as np

from . import constants, extend_border, window, window_stats, ssim_terms

#: Linear BT.709 / sRGB RGB to CIE XYZ (D65).
RGB_TO_XYZ = np.array([[0.4124, 0.3576, 0.1805],
                       [0.2126, 0.7152, 0.0722],
                       [0.0193, 0.1192, 0.9505]])
#: D65 white in XYZ: the rows of RGB_TO_XYZ summed (RGB = 1, 1, 1).
WHITE = RGB_TO_XYZ.sum(axis=1)
#: XYZ to the opponent planes (Q1, Q2, Q3) and back, as the section prints them.
XYZ_TO_OPP = np.array([[0.279, 0.72, -0.107],
                       [-0.449, 0.29, -0.077],
                       [0.086, -0.59, 0.501]])
OPP_TO_XYZ = np.array([[0.6204, -1.8704, -0.1553],
                       [1.3661, 0.9316, 0.4339],
                       [1.5013, 1.4176, 2.5331]])


def _apply(m, planes):
    return [m[i, 0] * planes[0] + m[i, 1] * planes[1] + m[i, 2] * planes[2] for i in range(3)]


def smooth_same(img, k: int = 11, sigma: float = 1.5) -> np.ndarray:
    """Gaussian smoothing with one output per pixel: the image extended by
    mirroring (extend_border "reflect"), then the window-weighted mean at
    every valid position."""
    w = window("gaussian", k, sigma)
    a = extend_border(img, k, "reflect")
    st = window_stats(a, a, w, 1)
    return st["mu1"]


def _lab_f(t):
    d = 6.0 / 29.0
    return np.where(t > d ** 3, np.cbrt(t), t / (3 * d * d) + 4.0 / 29.0)


def xyz_to_lab(X, Y, Z):
    """CIE 1976 L*, a*, b* relative to WHITE."""
    fx, fy, fz = _lab_f(X / WHITE[0]), _lab_f(Y / WHITE[1]), _lab_f(Z / WHITE[2])
    return 116.0 * fy - 16.0, 500.0 * (fx - fy), 200.0 * (fy - fz)


def cmssim_lab(r, g, b, k: int = 11, sigma: float = 1.5):
    """RGB planes in [0, 1] -> (L*, a*, b*) after the chromatic smoothing."""
    rgb = [np.asarray(t, dtype=np.float64) for t in (r, g, b)]
    xyz = _apply(RGB_TO_XYZ, rgb)
    q1, q2, q3 = _apply(XYZ_TO_OPP, xyz)
    q2, q3 = smooth_same(q2, k, sigma), smooth_same(q3, k, sigma)
    X, Y, Z = _apply(OPP_TO_XYZ, [q1, q2, q3])
    return xyz_to_lab(X, Y, Z)


def cmssim(rgb_x, rgb_y, k: int = 11, sigma: float = 1.5, K1: float = 0.01, K2: float = 0.03):
    """CMSSIM of one pair of RGB images ((R, G, B) planes in [0, 1]).
    Returns (score, weighted map, Delta E map)."""
    lx = cmssim_lab(*rgb_x, k=k, sigma=sigma)
    ly = cmssim_lab(*rgb_y, k=k, sigma=sigma)
    de = np.sqrt((lx[0] - ly[0]) ** 2 + (lx[1] - ly[1]) ** 2 + (lx[2] - ly[2]) ** 2)
    C1, C2 = constants(K1, K2, 100.0)
    st = window_stats(lx[0], ly[0], window("gaussian", k, sigma), 1)
    _, _, q = ssim_terms(st, C1, C2)
    c = (k - 1) // 2
    oh, ow = q.shape
    wmap = q * (1.0 - de[c:c + oh, c:c + ow] / 45.0)
    return float(wmap.mean()), wmap, de
