"""GPU parity of the scale handling: Z x Z block-mean downscaling
(gbssim_downscale) and MS-SSIM over the 9/7 wavelet pyramid
(GBSSIM_FLAG_PYRAMID_97), against oracle/scales.py and the oracle's
MS-SSIM with pyramid="97"."""
import numpy as np
import pytest
import torch

import oracle
from oracle import scales as S

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


@pytest.mark.parametrize("z", [1, 2, 3, 4, 7])
@pytest.mark.parametrize("dtype", [torch.uint8, torch.float32])
def test_downscale_matches_oracle(g, z, dtype):
    from paper_2101_06354_gb300 import synth

    x, _ = synth.luma_pairs_u8(3, 101, 133)
    if dtype == torch.float32:
        x = x.float() / 255
    got = g.downscale(x.to(DEV), z).cpu().double().numpy()
    for i in range(3):
        ref = S.downscale_block(x[i].double().numpy(), z)
        assert got[i].shape == ref.shape
        assert np.abs(got[i] - ref).max() <= 1e-6 * max(1.0, np.abs(ref).max())


def test_downscale_then_ssim_at_the_factor(g):
    """The recommended implementation's flow on a 1080p pair: Z from the
    round-min rule (4), block means, then SSIM of the downscaled pair."""
    from paper_2101_06354_gb300 import synth

    x, y = synth.luma_pairs_u8(1, 1080, 1920)
    z = g.downscale_factor(1080, 1920)
    assert z == 4
    xs, ys = g.downscale(x.to(DEV), z), g.downscale(y.to(DEV), z)
    got = g.ssim(xs, ys).item()
    ref, _ = oracle.ssim(S.downscale_block(x[0].numpy(), z), S.downscale_block(y[0].numpy(), z))
    assert abs(got - ref) <= 1e-6


@pytest.mark.parametrize("h,w", [(200, 232), (181, 203)])
def test_msssim_97_pyramid_matches_oracle(g, h, w):
    from paper_2101_06354_gb300 import synth

    x, y = synth.luma_pairs_u8(2, h, w)
    got = g.msssim(x.to(DEV), y.to(DEV), pyramid="97").cpu().numpy()
    for i in range(2):
        ref, _ = oracle.msssim(x[i].numpy(), y[i].numpy(), pyramid="97")
        assert abs(got[i] - ref) <= 1e-6
    avg = g.msssim(x.to(DEV), y.to(DEV)).cpu().numpy()
    assert np.all(np.abs(avg - got) > 0)  # a different pyramid gives a different score


def test_msssim_97_float_three_scales(g):
    from paper_2101_06354_gb300 import synth

    x, y = synth.loss_pairs_float(1, 2, 150, 170)
    xs, ys = x.reshape(2, 150, 170), y.reshape(2, 150, 170)
    kw = dict(L=1.0, scales=3, exponents=(0.3, 0.3, 0.4))
    got = g.msssim(xs.to(DEV), ys.to(DEV), pyramid="97", **kw).cpu().numpy()
    for i in range(2):
        ref, _ = oracle.msssim(xs[i].double().numpy(), ys[i].double().numpy(), pyramid="97", **kw)
        assert abs(got[i] - ref) <= 1e-6


def test_97_pyramid_rejected_where_unsupported(g):
    x = torch.zeros((1, 200, 200), device=DEV)
    with pytest.raises(g.GbssimError) as e:
        g.ssim_backward(x, x, multiscale=True, flags=g.FLAG_PYRAMID_97)
    assert e.value.status == g.ERR_UNSUPPORTED


def _rgb(n, h, w, seed):
    from paper_2101_06354_gb300 import synth

    planes = [synth.luma_pairs_u8(n, h, w, seed_ref=seed + c, seed_dist=seed + 10 + c) for c in range(3)]
    ref = tuple(p[0] for p in planes)
    dis = tuple(p[1] for p in planes)
    return ref, dis


@pytest.mark.parametrize("dtype", [torch.uint8, torch.float32])
def test_rgb_to_ycbcr_matches_oracle(g, dtype):
    ref, _ = _rgb(2, 37, 53, 5)
    if dtype == torch.float32:
        ref = tuple(t.float() / 255 for t in ref)
    y, cb, cr = g.rgb_to_ycbcr(*(t.to(DEV) for t in ref))
    ry, rcb, rcr = S.rgb_to_ycbcr(*(t.double().numpy() for t in ref))
    scale = 255.0 if dtype == torch.uint8 else 1.0
    for got, want in ((y, ry), (cb, rcb), (cr, rcr)):
        assert np.abs(got.cpu().double().numpy() - want).max() <= 2e-7 * scale * 4


@pytest.mark.parametrize("weights", [(0.8, 0.1, 0.1), (1.0, -0.3, -0.3)])
def test_colour_ssim_matches_oracle(g, weights):
    ref, dis = _rgb(3, 90, 120, 9)
    fr, ps, vid = g.colour_ssim(tuple(t.to(DEV) for t in ref), tuple(t.to(DEV) for t in dis), weights=weights)
    for t in range(3):
        rr = S.rgb_to_ycbcr(*(c[t].double().numpy() for c in ref))
        dd = S.rgb_to_ycbcr(*(c[t].double().numpy() for c in dis))
        s = [oracle.ssim(a, b)[0] for a, b in zip(rr, dd)]
        assert np.abs(ps[:, t].cpu().numpy() - s).max() <= 1e-5  # fp32 planes vs fp64
        assert abs(fr[t].item() - oracle.colour_score(*s, weights=weights)) <= 1e-5 / abs(sum(weights)) * 3
    assert abs(vid[0].item() - fr.mean().item()) <= 1e-12


# ---------------------------------------------------------------- border extension

@pytest.mark.parametrize("border", ["zero", "reflect"])
@pytest.mark.parametrize("h,w,kw", [
    (120, 150, {}),                                          # Gaussian 11, uint8: the fused kernel on extended planes
    (7, 9, {}),                                              # smaller than the window
    (97, 131, dict(window="box", k=8, stride=4)),            # exact integer box path
    (64, 70, dict(window="gaussian", k=7, sigma=1.0, stride=2)),  # generic path, strided
])
def test_ssim_border_matches_oracle(g, border, h, w, kw):
    from paper_2101_06354_gb300 import synth

    x, y = synth.single_pair_u8(h, w, seed_ref=h, seed_noise=w)
    mean, q = g.ssim(x.to(DEV), y.to(DEV), return_map=True, border=border, **kw)
    okw = dict(kw)
    okw["window_kind"] = okw.pop("window", "gaussian")
    ref_mean, ref = oracle.ssim(x.numpy(), y.numpy(), border=border, **okw)
    assert q.shape[1:] == ref["q"].shape
    assert np.abs(q[0].double().cpu().numpy() - ref["q"]).max() <= 1e-5
    assert abs(mean[0].item() - ref_mean) <= 1e-6


@pytest.mark.parametrize("border", ["zero", "reflect"])
def test_ssim_border_float_batch(g, border):
    from paper_2101_06354_gb300 import synth

    x, y = synth.luma_pairs_u8(3, 90, 101)
    xf, yf = x.float() / 255, y.float() / 255
    mean, q = g.ssim(xf.to(DEV), yf.to(DEV), return_map=True, border=border, L=1.0)
    for i in range(3):
        ref_mean, ref = oracle.ssim(xf[i].numpy(), yf[i].numpy(), border=border, L=1.0)
        assert np.abs(q[i].double().cpu().numpy() - ref["q"]).max() <= 1e-5
        assert abs(mean[i].item() - ref_mean) <= 1e-6


@pytest.mark.parametrize("border", ["zero", "reflect"])
@pytest.mark.parametrize("pyramid", ["avg2", "97"])
def test_msssim_border_matches_oracle(g, border, pyramid):
    from paper_2101_06354_gb300 import synth

    x, y = synth.luma_pairs_u8(2, 150, 171)
    s, per = g.msssim(x.to(DEV), y.to(DEV), per_scale=True, border=border, pyramid=pyramid)
    for i in range(2):
        ref, ref_per = oracle.msssim(x[i].numpy(), y[i].numpy(), border=border, pyramid=pyramid)
        assert abs(s[i].item() - ref) <= 1e-6
        np.testing.assert_allclose(per[i].cpu().numpy(), np.array(ref_per), rtol=0, atol=1e-6)


def test_border_rejected_where_unsupported(g):
    x = torch.zeros((1, 64, 64), dtype=torch.uint8, device=DEV)
    with pytest.raises(g.GbssimError) as e:
        g.SSIMLoss(border="zero")(x.float(), x.float().requires_grad_(True)).backward()
    assert e.value.status == g.ERR_UNSUPPORTED


@pytest.mark.parametrize("h,w,z", [(1080, 1920, None), (300, 420, 1), (512, 640, 2)])
def test_enhanced_ssim_matches_oracle(g, h, w, z):
    """Enhanced SSIM: z x z downscaling, 11 x 11 rectangular windows at
    stride 5, CoV pooling; against the oracle's composition of the same
    steps."""
    from oracle import pooling as P
    from paper_2101_06354_gb300 import synth

    x, y = synth.luma_pairs_u8(2, h, w)
    score, q = g.enhanced_ssim(x.to(DEV), y.to(DEV), z=z, return_map=True)
    zz = z if z is not None else S.downscale_factor(h, w)
    for i in range(2):
        a, b = x[i].numpy(), y[i].numpy()
        if zz > 1:
            a, b = S.downscale_block(a, zz), S.downscale_block(b, zz)
        _, ref = oracle.ssim(a, b, window_kind="box", k=11, stride=5)
        assert np.abs(q[i].double().cpu().numpy() - ref["q"]).max() <= 1e-5
        assert abs(score[i].item() - P.cov(ref["q"])) <= 1e-6


# ---------------------------------------------------------------- CMSSIM

def _rgb_pair(n, h, w, seed):
    from paper_2101_06354_gb300 import synth

    xs, ys = [], []
    for c in range(3):
        x, y = synth.luma_pairs_u8(n, h, w, seed_ref=seed + 10 * c, seed_dist=seed + 10 * c + 500)
        xs.append(x)
        ys.append(y)
    return xs, ys


@pytest.mark.parametrize("n,h,w,dtype,kw", [(2, 96, 130, torch.uint8, {}), (1, 64, 77, torch.float32, {}),
                                            (1, 80, 90, torch.uint8, dict(k=7, sigma=1.0, stride=2))])
def test_cmssim_matches_oracle(g, n, h, w, dtype, kw):
    from oracle import colour as C

    xs, ys = _rgb_pair(n, h, w, seed=h)
    if dtype == torch.float32:
        xs, ys = [t.float() / 255 for t in xs], [t.float() / 255 for t in ys]
    score, wmap = g.cmssim([t.to(DEV) for t in xs], [t.to(DEV) for t in ys], return_map=True, **kw)
    k, sigma, stride = kw.get("k", 11), kw.get("sigma", 1.5), kw.get("stride", 1)
    for i in range(n):
        fx = [t[i].double().numpy() / (255.0 if dtype == torch.uint8 else 1.0) for t in xs]
        fy = [t[i].double().numpy() / (255.0 if dtype == torch.uint8 else 1.0) for t in ys]
        if stride == 1:
            ref, rmap, _ = C.cmssim(fx, fy, k=k, sigma=sigma)
            assert np.abs(wmap[i].double().cpu().numpy() - rmap).max() <= 1e-5
            assert abs(score[i].item() - ref) <= 1e-6
        else:
            _, rmap, _ = C.cmssim(fx, fy, k=k, sigma=sigma)
            np.testing.assert_allclose(wmap[i].double().cpu().numpy(), rmap[::stride, ::stride], rtol=0, atol=1e-5)


def test_cmssim_identity_is_one(g):
    xs, _ = _rgb_pair(1, 70, 80, seed=3)
    d = [t.to(DEV) for t in xs]
    assert abs(g.cmssim(d, d).item() - 1.0) <= 1e-6
