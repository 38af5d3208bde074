"""Pins of the CMSSIM oracle (oracle/colour.py, Section "CMSSIM")."""
import numpy as np
import pytest

import oracle
from oracle import colour as C


def test_printed_opponent_matrices_invert_each_other():
    # the section prints both matrices rounded to 3-4 digits
    np.testing.assert_allclose(C.OPP_TO_XYZ @ C.XYZ_TO_OPP, np.eye(3), atol=5e-3)
    np.testing.assert_allclose(np.linalg.inv(C.XYZ_TO_OPP), C.OPP_TO_XYZ, atol=1e-2)


def test_rgb_to_xyz_is_bt709_d65():
    # the Y row is the BT.709 luma; white maps to the D65 white point
    np.testing.assert_allclose(C.RGB_TO_XYZ[1], [0.2126, 0.7152, 0.0722])
    np.testing.assert_allclose(C.WHITE, [0.9505, 1.0, 1.089], atol=1e-12)
    np.testing.assert_allclose(C.WHITE[0] / C.WHITE[1], 0.95047, atol=1e-4)


def test_cielab_closed_forms():
    L, a, b = C.xyz_to_lab(*[np.array([v]) for v in C.WHITE])
    np.testing.assert_allclose([L[0], a[0], b[0]], [100.0, 0.0, 0.0], atol=1e-12)
    L, a, b = C.xyz_to_lab(np.zeros(1), np.zeros(1), np.zeros(1))
    np.testing.assert_allclose([L[0], a[0], b[0]], [0.0, 0.0, 0.0], atol=1e-12)
    # grey: a* = b* = 0 and L* = 116 (Y)^(1/3) - 16 above the linear segment
    for yv in (0.18, 0.5):
        L, a, b = C.xyz_to_lab(*[np.array([yv * w]) for w in C.WHITE])
        assert L[0] == pytest.approx(116 * yv ** (1 / 3) - 16, abs=1e-12)
        assert abs(a[0]) < 1e-12 and abs(b[0]) < 1e-12
    # the two branches of f meet at (6/29)^3
    t = (6 / 29) ** 3
    assert C._lab_f(np.array([t * (1 + 1e-12)]))[0] == pytest.approx(C._lab_f(np.array([t]))[0], abs=1e-9)


def test_smoothing_keeps_constants_and_sums():
    a = np.full((20, 25), 0.3)
    np.testing.assert_allclose(C.smooth_same(a), a, rtol=1e-13)
    r = np.random.default_rng(3).uniform(size=(30, 40))
    s = C.smooth_same(r)
    assert s.shape == r.shape
    # interior: the plain window mean
    np.testing.assert_allclose(s[5:-5, 5:-5], oracle.window_stats(r, r, oracle.window("gaussian", 11, 1.5))["mu1"],
                               rtol=0, atol=1e-13)


def test_cmssim_identity_and_constant_colour_closed_form():
    r = np.random.default_rng(4)
    x = [r.uniform(size=(40, 48)) for _ in range(3)]
    s, wmap, de = C.cmssim(x, x)
    assert s == pytest.approx(1.0, abs=1e-12) and np.abs(de).max() == 0.0
    # two uniform colours: sigma = 0 so cs = 1, l from the L* values, and a constant Delta E
    cx, cy = (0.6, 0.3, 0.2), (0.5, 0.35, 0.25)
    xs = [np.full((30, 30), v) for v in cx]
    ys = [np.full((30, 30), v) for v in cy]
    s, wmap, de = C.cmssim(xs, ys)
    lx = C.xyz_to_lab(*[np.array([v]) for v in (C.RGB_TO_XYZ @ np.array(cx))])
    ly = C.xyz_to_lab(*[np.array([v]) for v in (C.RGB_TO_XYZ @ np.array(cy))])
    # the chromatic smoothing of constants changes nothing, so the opponent
    # round trip is the printed matrices' product applied to XYZ
    def lab_rt(c):
        xyz = C.OPP_TO_XYZ @ (C.XYZ_TO_OPP @ (C.RGB_TO_XYZ @ np.array(c)))
        return [v[0] for v in C.xyz_to_lab(*[np.array([t]) for t in xyz])]
    Lx, ax, bx = lab_rt(cx)
    Ly, ay, by = lab_rt(cy)
    d = np.sqrt((Lx - Ly) ** 2 + (ax - ay) ** 2 + (bx - by) ** 2)
    C1, _ = oracle.constants(L=100.0)
    l = (2 * Lx * Ly + C1) / (Lx ** 2 + Ly ** 2 + C1)
    assert s == pytest.approx(l * (1 - d / 45), rel=1e-9)
    np.testing.assert_allclose(de, d, rtol=1e-9)
    assert abs(lx[0][0] - Lx) < 1.0  # the round trip moves L* only by the matrices' rounding
