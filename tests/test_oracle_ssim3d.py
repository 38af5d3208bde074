"""Pins of the SSIM-3D oracle (Section "Spatio-Temporal SSIM"): window sums
against numpy's sliding windows, reduction to the 2-D box SSIM for kt = 1 and
for a static video, closed forms and invariants."""
import numpy as np
import pytest
from numpy.lib.stride_tricks import sliding_window_view

import oracle


def _video(T=7, H=23, W=29, seed=0):
    r = np.random.default_rng(seed)
    x = r.integers(0, 256, (T, H, W), dtype=np.uint8)
    y = np.clip(x.astype(int) + r.integers(-30, 31, x.shape), 0, 255).astype(np.uint8)
    return x, y


@pytest.mark.parametrize("k,kt", [(5, 3), (11, 1), (3, 7), (1, 2)])
def test_sums_equal_sliding_windows(k, kt):
    x, y = _video(T=8, H=14, W=17, seed=k + kt)
    got = oracle.box3d_sums(x, y, k, kt)
    xi, yi = x.astype(np.int64), y.astype(np.int64)
    for q, a in enumerate((xi, yi, xi * xi, yi * yi, xi * yi)):
        ref = sliding_window_view(a, (kt, k, k)).sum(axis=(-3, -2, -1))
        np.testing.assert_array_equal(got[..., q], ref)


def test_kt1_is_framewise_box_ssim():
    x, y = _video()
    _, frames, q = oracle.ssim3d(x, y, k=8, kt=1)
    for t in range(x.shape[0]):
        m2, q2, _, _ = oracle.box_ssim(x[t], y[t], k=8, stride=1)
        np.testing.assert_allclose(q[t], q2, rtol=0, atol=1e-13)
        assert frames[t] == pytest.approx(m2, abs=1e-13)


def test_static_video_is_the_2d_score():
    x, y = _video(T=1)
    xs, ys = np.repeat(x, 6, axis=0), np.repeat(y, 6, axis=0)
    score, frames, _ = oracle.ssim3d(xs, ys, k=11, kt=4)
    m2, _, _, _ = oracle.box_ssim(x[0], y[0], k=11, stride=1)
    assert frames.shape == (3,)
    np.testing.assert_allclose(frames, m2, rtol=0, atol=1e-12)
    assert score == pytest.approx(m2, abs=1e-12)


def test_identity_constant_and_shapes():
    x, _ = _video()
    s, frames, q = oracle.ssim3d(x, x, k=5, kt=3)
    assert s == 1.0 and np.all(q == 1.0) and frames.shape == (5,)
    a, b = 100, 110
    xc = np.full((5, 15, 15), a, np.uint8)
    yc = np.full((5, 15, 15), b, np.uint8)
    C1, _ = oracle.constants()
    _, _, q = oracle.ssim3d(xc, yc, k=11, kt=2)
    np.testing.assert_allclose(q, (2 * a * b + C1) / (a * a + b * b + C1), rtol=1e-12)


def test_msssim3d_one_scale_is_ssim3d():
    x, y = _video(T=6, H=30, W=33, seed=4)
    s3, f3, _ = oracle.ssim3d(x, y, k=5, kt=3)
    s, f, per = oracle.msssim3d(x, y, k=5, kt=3, scales=1, exponents=(1.0,))
    np.testing.assert_allclose(f, f3, rtol=0, atol=1e-12)
    assert s == pytest.approx(s3, abs=1e-12)


def test_msssim3d_kt1_is_framewise_msssim_with_box_window():
    x, y = _video(T=3, H=60, W=70, seed=5)
    _, frames, _ = oracle.msssim3d(x, y, k=5, kt=1, scales=3, exponents=(0.3, 0.3, 0.4))
    for t in range(3):
        ref, _ = oracle.msssim(x[t], y[t], scales=3, exponents=(0.3, 0.3, 0.4), window_kind="box", k=5)
        assert frames[t] == pytest.approx(ref, abs=1e-12)


def test_msssim3d_identity_and_static_video():
    x, y = _video(T=1, H=64, W=72, seed=6)
    xs, ys = np.repeat(x, 4, axis=0), np.repeat(y, 4, axis=0)
    s, frames, _ = oracle.msssim3d(xs, ys, k=5, kt=2, scales=3, exponents=(0.3, 0.3, 0.4))
    ref, _ = oracle.msssim(x[0], y[0], scales=3, exponents=(0.3, 0.3, 0.4), window_kind="box", k=5)
    np.testing.assert_allclose(frames, ref, rtol=0, atol=1e-12)
    s1, _, _ = oracle.msssim3d(xs, xs, k=5, kt=2, scales=3, exponents=(0.3, 0.3, 0.4))
    assert s1 == pytest.approx(1.0, abs=1e-12)
