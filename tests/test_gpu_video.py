"""GPU parity of colour + temporal pooling (gbssim_video) against the oracle:
per-plane SSIM at each plane's own resolution, the 6:1:1 (and other) channel
weights, the temporal mean, the 10th percentile and percentile pooling."""
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


@pytest.mark.parametrize("frames,h,w,weights,pct,r", [(12, 150, 200, (6, 1, 1), 10.0, 4.0),
                                                      (7, 96, 130, (0.8, 0.1, 0.1), 25.0, 2.0),
                                                      (1, 64, 64, (1.0, -0.3, -0.3), 10.0, 1.0),
                                                      (33, 48, 66, (6, 1, 1), 0.0, 3.0)])
def test_video_matches_oracle(g, frames, h, w, weights, pct, r):
    from paper_2101_06354_gb300 import synth

    v = synth.video_yuv420_u8(frames, h, w)
    xs = [v[p][0].to(DEV) for p in "yuv"]
    ys = [v[p][1].to(DEV) for p in "yuv"]
    fr, ps, vid = g.video_ssim(xs, ys, weights=weights, percentile=pct, pp_r=r)
    fr, ps, vid = fr.cpu().numpy(), ps.cpu().numpy(), vid.cpu().numpy()
    ref_planes = np.zeros((3, frames))
    for q, name in enumerate("yuv"):
        for t in range(frames):
            ref_planes[q, t], _ = oracle.ssim(v[name][0][t].numpy(), v[name][1][t].numpy())
    ref_frames = np.array([oracle.colour_score(*ref_planes[:, t], weights=weights) for t in range(frames)])
    np.testing.assert_allclose(ps, ref_planes, rtol=0, atol=1e-6)
    np.testing.assert_allclose(fr, ref_frames, rtol=0, atol=1e-6)
    m, pv, pp = oracle.temporal_pool(ref_frames, pct, r=r)
    assert abs(vid[0] - m) <= 1e-6 and abs(vid[1] - pv) <= 1e-6 and abs(vid[2] - pp) <= 1e-6
    # the pooled values are exact functions of the frame scores the GPU produced
    m2, pv2, pp2 = oracle.temporal_pool(fr, pct, r=r)
    assert abs(vid[0] - m2) <= 1e-12 and abs(vid[1] - pv2) <= 1e-12 and abs(vid[2] - pp2) <= 1e-12


def test_video_4k_sampled_frames(g):
    """The 4K YUV420 workload shape (3840x2160 luma) for a few frames, checked
    frame by frame against the oracle."""
    from paper_2101_06354_gb300 import synth

    v = synth.video_yuv420_u8(4, 2160, 3840, device=DEV)
    xs = [v[p][0] for p in "yuv"]
    ys = [v[p][1] for p in "yuv"]
    fr, ps, vid = g.video_ssim(xs, ys)
    for t in (0, 3):
        ref = [oracle.ssim(v[p][0][t].cpu().numpy(), v[p][1][t].cpu().numpy())[0] for p in "yuv"]
        assert abs(fr[t].item() - oracle.colour_score(*ref)) <= 1e-6
