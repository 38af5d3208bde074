"""GPU parity of SSIM-3D (gbssim_ssim3d, Section "Spatio-Temporal SSIM")
against the FP64 oracle's direct k x k x kt window sums.  The GPU window sums
are exact integers, so only the final fp32 formula rounds: maps within 1e-5
per element, frame and video means within 1e-6."""
import numpy as np
import pytest
import torch

import oracle

pytestmark = pytest.mark.gpu
DEV = "cuda"


@pytest.fixture(scope="module")
def g():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2101_06354_gb300 import build

    build.build()
    from paper_2101_06354_gb300 import gbssim

    return gbssim


def _video(T, H, W, seed=0):
    from paper_2101_06354_gb300 import synth

    v = synth.video_yuv420_u8(T, H, W, seeds=(seed, seed + 1, seed + 2))
    return v["y"][0].contiguous(), v["y"][1].contiguous()


@pytest.mark.parametrize("T,H,W,k,kt", [(9, 40, 70, 11, 5), (6, 33, 150, 5, 3), (4, 26, 64, 11, 1),
                                        (12, 20, 21, 3, 12), (7, 80, 129, 8, 4),
                                        (10, 40, 100, 31, 9),   # N = 8649: int64 window sums
                                        (20, 24, 40, 3, 2), (16, 30, 50, 5, 3),  # few tiles: frames split over CTAs
                                        (6, 64, 128, 31, 2), (5, 50, 160, 19, 3),  # 16-byte rows: bulk-copied tiles
                                        # k = 11 on 16-byte rows: the register-column kernel (ragged tiles,
                                        # kt = 1, few tiles with the frames split over CTAs)
                                        (9, 40, 80, 11, 5), (7, 70, 144, 11, 3), (5, 27, 64, 11, 1),
                                        (30, 26, 64, 11, 2), (11, 37, 208, 11, 11)])
def test_ssim3d_matches_oracle(g, T, H, W, k, kt):
    x, y = _video(T, H, W, seed=T + k)
    score, frames, q = g.ssim3d(x.to(DEV), y.to(DEV), kt=kt, k=k, return_map=True)
    rs, rf, rq = oracle.ssim3d(x.numpy(), y.numpy(), k=k, kt=kt)
    assert q.shape == rq.shape
    assert np.abs(q.double().cpu().numpy() - rq).max() <= 1e-5
    assert np.abs(frames.cpu().numpy() - rf).max() <= 1e-6
    assert abs(score.item() - rs) <= 1e-6


def test_kt1_equals_framewise_box_ssim(g):
    x, y = _video(5, 60, 96, seed=3)
    _, frames, q = g.ssim3d(x.to(DEV), y.to(DEV), kt=1, k=8, return_map=True)
    m2, q2 = g.ssim(x.to(DEV), y.to(DEV), return_map=True, window="box", k=8, stride=1)
    assert torch.allclose(q, q2, rtol=0, atol=1e-6)
    assert torch.allclose(frames, m2, rtol=0, atol=1e-6)


def test_ssim3d_full_hd_sampled(g):
    """1080p, 10 frames, kt = 5: sampled output positions against the oracle
    on the crop that holds their window (the window is local)."""
    x, y = _video(10, 1080, 1920, seed=7)
    k, kt = 11, 5
    score, frames, q = g.ssim3d(x.to(DEV), y.to(DEV), kt=kt, k=k, return_map=True)
    qc = q.cpu().numpy()
    r = np.random.default_rng(1)
    for _ in range(40):
        t, a, b = r.integers(0, 10 - kt + 1), r.integers(0, 1070), r.integers(0, 1910)
        xs = x[t:t + kt, a:a + k, b:b + k].numpy()
        ys = y[t:t + kt, a:a + k, b:b + k].numpy()
        _, _, rq = oracle.ssim3d(xs, ys, k=k, kt=kt)
        assert abs(qc[t, a, b] - rq[0, 0, 0]) <= 1e-5
    assert abs(score.item() - frames.mean().item()) <= 1e-12
    assert torch.isfinite(q).all()


def test_ssim3d_rejects_unsupported(g):
    x = torch.zeros((4, 32, 32), dtype=torch.uint8, device=DEV)
    with pytest.raises(g.GbssimError) as e:
        g.ssim3d(x, x, kt=5)                      # kt > T
    assert e.value.status == g.ERR_TOO_SMALL
    with pytest.raises(g.GbssimError) as e:
        g.ssim3d(x, x, kt=2, k=11, stride=2)      # spatial stride
    assert e.value.status == g.ERR_UNSUPPORTED


# ---------------------------------------------------------------- MS-SSIM-3D

@pytest.mark.parametrize("T,H,W,k,kt,scales,combine", [
    (6, 96, 136, 5, 3, 3, "product"),   # every level's width a multiple of 4: vector loads
    (5, 97, 131, 5, 2, 3, "sum"),       # odd sizes: floor halving, scalar loads on the upper levels
    (4, 176, 200, 11, 2, 4, "product"),
    (3, 248, 256, 31, 3, 4, "product"),  # largest window
    (7, 70, 90, 3, 7, 2, "sum"),        # one output frame
    (14, 64, 72, 3, 2, 3, "product"),   # frames split over CTAs on every level
])
def test_msssim3d_matches_oracle(g, T, H, W, k, kt, scales, combine):
    x, y = _video(T, H, W, seed=T + k + scales)
    exps = tuple(oracle.MSSSIM_EXPONENTS[:scales]) if scales == 5 else tuple([1.0 / scales] * scales)
    score, frames, per = g.msssim3d(x.to(DEV), y.to(DEV), kt=kt, k=k, scales=scales, exponents=exps,
                                    combine=combine, per_scale=True)
    rs, rf, rper = oracle.msssim3d(x.numpy(), y.numpy(), k=k, kt=kt, scales=scales, exponents=exps, combine=combine)
    pc = per.cpu().numpy()
    for j in range(scales):
        assert np.abs(pc[:, j, :] - rper[j]).max() <= 1e-6, j
    assert np.abs(frames.cpu().numpy() - rf).max() <= 1e-6
    assert abs(score.item() - rs) <= 1e-6


def test_msssim3d_one_scale_equals_ssim3d(g):
    x, y = _video(8, 120, 200, seed=11)
    s3, f3 = g.ssim3d(x.to(DEV), y.to(DEV), kt=4, k=11)
    s, f = g.msssim3d(x.to(DEV), y.to(DEV), kt=4, k=11, scales=1, exponents=(1.0,), combine="sum")
    assert torch.equal(f, f3)
    assert s.item() == s3.item()


def test_msssim3d_full_hd_kt1_is_framewise_box_msssim(g):
    """1080p, 4 frames, kt = 1: every frame's MS-SSIM-3D is the frame's
    MS-SSIM with the k x k box window (the same statistics, another kernel)."""
    x, y = _video(4, 1080, 1920, seed=12)
    xd, yd = x.to(DEV), y.to(DEV)
    _, f = g.msssim3d(xd, yd, kt=1, k=8, scales=5)
    ref = g.msssim(xd, yd, window="box", k=8, scales=5)
    assert torch.allclose(f, ref, rtol=0, atol=1e-6)
    s, f5 = g.msssim3d(xd, yd, kt=3, k=8, scales=5)
    assert torch.isfinite(f5).all() and f5.shape == (2,)
    assert abs(s.item() - f5.mean().item()) <= 1e-12


def test_msssim3d_rejects_unsupported(g):
    x = torch.zeros((4, 64, 64), dtype=torch.uint8, device=DEV)
    with pytest.raises(g.GbssimError) as e:
        g.msssim3d(x, x, kt=2, k=32, scales=2, exponents=(0.5, 0.5))   # windows up to 31 x 31
    assert e.value.status == g.ERR_UNSUPPORTED
    with pytest.raises(g.GbssimError) as e:
        g.msssim3d(x, x, kt=2, k=11, scales=4, exponents=(0.25,) * 4)  # level 3 is 8 x 8 (64 >> 3)
    assert e.value.status == g.ERR_TOO_SMALL
    with pytest.raises(g.GbssimError) as e:
        g.msssim3d(x, x, kt=5, k=5, scales=2, exponents=(0.5, 0.5))    # kt > T
    assert e.value.status == g.ERR_TOO_SMALL
