"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances: |dQ| <= 1e-5 per map element and |d score| <= 1e-6 per pooled
score (SSIM, per-scale MS-SSIM terms and the MS-SSIM score); integer window
sums bit-exact.  Sizes span several CTA tiles and ragged tails; inputs are
the seeded synthetic workloads plus adversarial patterns (step edges,
impulses, flat bands at 0 and 255) that break a naive fp32 variance.
"""
import numpy as np
import pytest
import torch

import oracle

pytestmark = pytest.mark.gpu

MAP_TOL = 1e-5
POOL_TOL = 1e-6


@pytest.fixture(scope="module")
def g():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2101_06354_gb300 import build

    build.build()
    from paper_2101_06354_gb300 import gbssim

    return gbssim


@pytest.fixture(scope="module")
def synth():
    from paper_2101_06354_gb300 import synth as s

    return s


DEV = "cuda"


def _np(t):
    return t.detach().float().cpu().numpy() if t.dtype != torch.uint8 else t.cpu().numpy()


def _adversarial(h, w, L, seed):
    r = np.random.default_rng(seed)
    out = {}
    e = np.zeros((h, w)); e[h // 2:, :] = L
    out["hedge"] = (e, np.clip(e + r.integers(-1, 2, e.shape) * L / 255, 0, L))
    fl = np.zeros((h, w)); fl[:, : w // 3] = L; fl[:, 2 * w // 3:] = L
    out["flat_bands"] = (fl, np.clip(fl + r.integers(-1, 2, fl.shape) * L / 255, 0, L))
    imp = np.full((h, w), L); imp[::9, ::7] = 0
    out["impulse"] = (imp, np.round(imp * 0.99 * 255 / L) * L / 255)
    cb = ((np.indices((h, w)) // 3).sum(0) % 2) * L
    out["checker"] = (cb, np.clip(cb + r.normal(0, 2 * L / 255, cb.shape), 0, L))
    return out


def _check_map(qmap, ref_q, tol=MAP_TOL):
    err = np.abs(qmap - ref_q).max()
    assert err <= tol, "max |dQ| = %g" % err


# --------------------------------------------------------------------------- SSIM, Gaussian 11

@pytest.mark.parametrize("h,w", [(256, 256), (300, 333), (11, 11), (12, 600), (600, 12), (150, 75), (91, 200),
                                 (11, 20011), (3000, 11)])
def test_ssim_u8_matches_oracle(g, synth, h, w):
    x, y = synth.single_pair_u8(h, w)
    mean, qmap = g.ssim(x.to(DEV), y.to(DEV), return_map=True)
    ref_mean, ref = oracle.ssim(x.numpy(), y.numpy())
    _check_map(qmap[0].cpu().numpy(), ref["q"])
    assert abs(mean[0].item() - ref_mean) <= POOL_TOL


@pytest.mark.parametrize("name", ["hedge", "flat_bands", "impulse", "checker"])
@pytest.mark.parametrize("L,dtype", [(255.0, torch.uint8), (1.0, torch.float32), (1.0, torch.float16),
                                     (1.0, torch.bfloat16)])
def test_ssim_adversarial(g, name, L, dtype):
    x, y = _adversarial(70, 150, L, 3)[name]
    xt = torch.tensor(x).to(dtype)
    yt = torch.tensor(y).to(dtype)
    mean, qmap = g.ssim(xt.to(DEV), yt.to(DEV), return_map=True, L=L)
    xr, yr = _np(xt).astype(np.float64), _np(yt).astype(np.float64)  # same rounded values
    ref_mean, ref = oracle.ssim(xr, yr, L=L)
    _check_map(qmap[0].cpu().numpy(), ref["q"])
    assert abs(mean[0].item() - ref_mean) <= POOL_TOL


@pytest.mark.parametrize("dtype", [torch.float32, torch.float16, torch.bfloat16])
def test_ssim_float_inputs_batch(g, synth, dtype):
    x, y = synth.loss_pairs_float(2, 2, 140, 130)
    xt, yt = x.to(dtype), y.to(dtype)
    mean, qmap = g.ssim(xt.to(DEV), yt.to(DEV), return_map=True, L=1.0)
    xr, yr = _np(xt).reshape(4, 140, 130), _np(yt).reshape(4, 140, 130)
    for i in range(4):
        ref_mean, ref = oracle.ssim(xr[i].astype(np.float64), yr[i].astype(np.float64), L=1.0)
        _check_map(qmap[i].cpu().numpy(), ref["q"])
        assert abs(mean[i].item() - ref_mean) <= POOL_TOL


def test_ssim_identity_and_symmetry(g, synth):
    x, y = synth.single_pair_u8(200, 220)
    xd, yd = x.to(DEV), y.to(DEV)
    m_same, q_same = g.ssim(xd, xd, return_map=True)
    assert np.abs(q_same.cpu().numpy() - 1.0).max() <= 1e-6
    assert abs(m_same.item() - 1.0) <= 1e-7
    a = g.ssim(xd, yd).item()
    b = g.ssim(yd, xd).item()
    assert abs(a - b) <= 1e-7


def test_ssim_strided_views_and_map_ld(g, synth):
    # row stride > width, image stride padded, map with ld > OW
    n, h, w = 3, 120, 140
    x, y = synth.luma_pairs_u8(n, h, w)
    bx = torch.zeros((n, h + 3, w + 20), dtype=torch.uint8)
    by = torch.zeros_like(bx)
    bx[:, :h, :w] = x
    by[:, :h, :w] = y
    xd, yd = bx.to(DEV)[:, :h, :w], by.to(DEV)[:, :h, :w]
    px, py = g.plane(xd), g.plane(yd)
    assert px.row_stride == w + 20 and px.image_stride == (h + 3) * (w + 20)
    p = g.make_params()
    ws = g.workspace(px, p, g.OP_SSIM, xd.device)
    oh, ow = h - 10, w - 10
    mp = torch.full((n, oh + 2, ow + 7), -7.0, device=DEV)
    mean = torch.empty(n, dtype=torch.float64, device=DEV)
    import ctypes
    rc = g.lib.gbssim_ssim_map(ctypes.byref(px), ctypes.byref(py), ctypes.byref(p), mp.data_ptr(), mp.stride(1),
                               mp.stride(0), mean.data_ptr(), ws.data_ptr(), ws.numel(),
                               torch.cuda.current_stream().cuda_stream)
    assert rc == 0
    mp = mp.cpu().numpy()
    for i in range(n):
        ref_mean, ref = oracle.ssim(x[i].numpy(), y[i].numpy())
        _check_map(mp[i, :oh, :ow], ref["q"])
        assert np.all(mp[i, oh:, :] == -7.0) and np.all(mp[i, :, ow:] == -7.0)
        assert abs(mean[i].item() - ref_mean) <= POOL_TOL


def test_ssim_deterministic(g, synth):
    x, y = synth.luma_pairs_u8(4, 300, 400)
    xd, yd = x.to(DEV), y.to(DEV)
    a = g.ssim(xd, yd)
    for _ in range(3):
        assert torch.equal(a, g.ssim(xd, yd))


# --------------------------------------------------------------------------- generic path (other k, stride)

@pytest.mark.parametrize("window,k,sigma,stride", [("gaussian", 7, 1.0, 1), ("gaussian", 11, 1.5, 2),
                                                   ("gaussian", 11, 1.5, 5), ("gaussian", 15, 2.0, 3),
                                                   ("box", 11, 1.5, 1), ("gaussian", 3, 0.7, 1),
                                                   ("gaussian", 21, 3.0, 4)])
@pytest.mark.parametrize("dtype", [torch.uint8, torch.float32])
def test_ssim_generic_windows_and_strides(g, synth, window, k, sigma, stride, dtype):
    if window == "box" and dtype == torch.uint8:
        pytest.skip("uint8 box windows take the integer path (tested below)")
    x, y = synth.single_pair_u8(97, 133)
    xt, yt = x.to(dtype), y.to(dtype)
    mean, qmap = g.ssim(xt.to(DEV), yt.to(DEV), return_map=True, window=window, k=k, sigma=sigma, stride=stride)
    ref_mean, ref = oracle.ssim(x.numpy(), y.numpy(), window, k, sigma, stride=stride)
    _check_map(qmap[0].cpu().numpy(), ref["q"])
    assert abs(mean[0].item() - ref_mean) <= POOL_TOL


# --------------------------------------------------------------------------- box / integral images

@pytest.mark.parametrize("k,s,h,w", [(8, 4, 270, 481), (8, 4, 300, 1024), (12, 4, 150, 768), (4, 4, 97, 512),
                                     (8, 4, 8, 8), (11, 1, 100, 130), (7, 3, 64, 100),
                                     (16, 8, 100, 200), (4, 4, 33, 70), (63, 1, 70, 80), (1, 1, 20, 20),
                                     (12, 4, 50, 90), (5, 2, 41, 77)])
def test_window_sums_bit_exact(g, synth, k, s, h, w):
    x, y = synth.single_pair_u8(h, w, seed_ref=5, seed_noise=6)
    got = g.window_sums(x.to(DEV), y.to(DEV), k, s)[0].cpu().numpy()
    ref = oracle.box_sums(x.numpy(), y.numpy(), k, s, "integral")
    assert got.shape == ref.shape
    np.testing.assert_array_equal(got, ref)


@pytest.mark.parametrize("flags", [0, 1])
@pytest.mark.parametrize("k,n,h,w", [(8, 3, 100, 160), (4, 2, 70, 64), (12, 2, 300, 1040), (8, 5, 1080, 1920)])
def test_window_sums_batched_aligned(g, synth, k, n, h, w, flags):
    """Batched, 16-byte aligned planes (vector loads, or with flags=1 the
    bulk-tensor-copy loader), widths below and above one 256-byte tile,
    ragged last tiles."""
    x, y = synth.luma_pairs_u8(n, h, w)
    got = g.window_sums(x.to(DEV), y.to(DEV), k, 4, flags=flags).cpu().numpy()
    for i in range(n):
        np.testing.assert_array_equal(got[i], oracle.box_sums(x[i].numpy(), y[i].numpy(), k, 4))


def test_window_sums_unaligned_and_extremes(g):
    # odd row stride forces the byte-gather path; 255 everywhere stresses int ranges
    x = torch.full((1, 40, 51), 255, dtype=torch.uint8)
    y = torch.zeros((1, 40, 51), dtype=torch.uint8)
    y[0, ::2] = 255
    for k, s in [(8, 4), (16, 4), (9, 1)]:
        got = g.window_sums(x.to(DEV), y.to(DEV), k, s)[0].cpu().numpy()
        np.testing.assert_array_equal(got, oracle.box_sums(x[0].numpy(), y[0].numpy(), k, s))


@pytest.mark.parametrize("k,s,w", [(8, 4, 210), (8, 4, 1024), (12, 4, 528), (4, 4, 1040), (11, 1, 210), (7, 3, 210),
                                   (16, 8, 210)])
def test_box_ssim_u8(g, synth, k, s, w):
    # widths that are multiples of 16 take the 16-byte vector path over several tile columns
    x, y = synth.luma_pairs_u8(2, 150, w)
    mean, qmap = g.ssim(x.to(DEV), y.to(DEV), return_map=True, window="box", k=k, stride=s)
    for i in range(2):
        ref_mean, ref_q, _, _ = oracle.box_ssim(x[i].numpy(), y[i].numpy(), k, s)
        _check_map(qmap[i].cpu().numpy(), ref_q)
        assert abs(mean[i].item() - ref_mean) <= POOL_TOL


@pytest.mark.parametrize("k", [4, 8, 12])
def test_box_ssim_tma_loader_matches(g, synth, k):
    x, y = synth.luma_pairs_u8(3, 333, 1040)
    a, ma = g.ssim(x.to(DEV), y.to(DEV), return_map=True, window="box", k=k, stride=4)
    b, mb = g.ssim(x.to(DEV), y.to(DEV), return_map=True, window="box", k=k, stride=4, flags=g.FLAG_BOX_TMA)
    assert torch.equal(ma, mb)
    # same map, pooled with different fp32 groupings (per-warp strips vs tiles)
    assert torch.allclose(a, b, rtol=0, atol=1e-7)
    ref_mean, ref_q, _, _ = oracle.box_ssim(x[1].numpy(), y[1].numpy(), k, 4)
    _check_map(mb[1].cpu().numpy(), ref_q)
    assert abs(a[1].item() - ref_mean) <= POOL_TOL


def test_box_ssim_adversarial(g):
    for name, (x, y) in _adversarial(64, 100, 255.0, 9).items():
        xt = torch.tensor(x).to(torch.uint8)
        yt = torch.tensor(y).to(torch.uint8)
        mean, qmap = g.ssim(xt.to(DEV), yt.to(DEV), return_map=True, window="box", k=8, stride=4)
        ref_mean, ref_q, _, _ = oracle.box_ssim(xt.numpy(), yt.numpy(), 8, 4)
        _check_map(qmap[0].cpu().numpy(), ref_q)


# --------------------------------------------------------------------------- pooling

def test_ssim_pool_mean(g, synth):
    x, y = synth.luma_pairs_u8(2, 200, 300)
    mean, qmap = g.ssim(x.to(DEV), y.to(DEV), return_map=True)
    pooled = g.ssim_pool(qmap)
    # the fused kernel pools with fp32 (Kahan) partial sums, well inside the 1e-6 bar
    assert torch.allclose(pooled, mean, rtol=0, atol=2e-7)
    ref = np.array([qmap[i].double().mean().item() for i in range(2)])
    assert np.abs(pooled.cpu().numpy() - ref).max() <= 1e-9


# --------------------------------------------------------------------------- MS-SSIM

@pytest.mark.parametrize("h,w", [(200, 232), (353, 277), (176, 176)])
def test_msssim_u8(g, synth, h, w):
    x, y = synth.luma_pairs_u8(2, h, w)
    score, per = g.msssim(x.to(DEV), y.to(DEV), per_scale=True)
    for i in range(2):
        ref_score, ref_per = oracle.msssim(x[i].numpy(), y[i].numpy())
        assert abs(score[i].item() - ref_score) <= POOL_TOL
        np.testing.assert_allclose(per[i].cpu().numpy(), np.array(ref_per), rtol=0, atol=POOL_TOL)


@pytest.mark.parametrize("dtype", [torch.uint8, torch.float32])
def test_msssim_score_same_with_and_without_per_scale(g, synth, dtype):
    """Without per-scale output the levels below the last form only the
    contrast-structure term (their mean Q is not pooled): the score is
    bit-identical to the run that forms and returns both, and the returned
    per-scale pairs match the oracle."""
    x, y = synth.luma_pairs_u8(3, 300, 420)
    if dtype != torch.uint8:
        x, y = x.to(dtype) / 255, y.to(dtype) / 255
    kw = {} if dtype == torch.uint8 else dict(L=1.0)
    alone = g.msssim(x.to(DEV), y.to(DEV), **kw)
    score, per = g.msssim(x.to(DEV), y.to(DEV), per_scale=True, **kw)
    assert torch.equal(alone, score)
    for i in (0, 2):
        _, ref_per = oracle.msssim(x[i].double().numpy(), y[i].double().numpy(), **kw)
        np.testing.assert_allclose(per[i].cpu().numpy(), np.array(ref_per), rtol=0, atol=POOL_TOL)


@pytest.mark.parametrize("kw", [dict(combine="sum"), dict(scales=3, exponents=(0.3, 0.3, 0.4)),
                                dict(window="box", k=8), dict(k=7, sigma=1.0), dict(stride=2),
                                dict(scales=1, exponents=(1.0,))])
def test_msssim_variants(g, synth, kw):
    x, y = synth.luma_pairs_u8(1, 260, 300)
    score, per = g.msssim(x.to(DEV), y.to(DEV), per_scale=True, **kw)
    okw = dict(kw)
    stride = okw.pop("stride", 1)
    if stride != 1:
        # the oracle's msssim has no stride: combine strided per-scale SSIM by hand
        exps = oracle.MSSSIM_EXPONENTS
        a, b = x[0].numpy().astype(float), y[0].numpy().astype(float)
        m = []
        for j in range(5):
            _, maps = oracle.ssim(a, b, stride=stride)
            m.append(maps["cs"].mean() if j < 4 else maps["q"].mean())
            a, b = oracle.downsample2x2(a), oracle.downsample2x2(b)
        ref = float(np.prod(np.power(m, exps)))
    else:
        if okw.get("window") == "box":
            okw["window_kind"] = okw.pop("window")
        ref, _ = oracle.msssim(x[0].numpy(), y[0].numpy(), **okw)
    assert abs(score[0].item() - ref) <= POOL_TOL


@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16])
def test_msssim_float(g, synth, dtype):
    x, y = synth.loss_pairs_float(1, 2, 256, 256)
    xt, yt = x.to(dtype), y.to(dtype)
    score = g.msssim(xt.to(DEV), yt.to(DEV), L=1.0)
    xr, yr = _np(xt).reshape(2, 256, 256), _np(yt).reshape(2, 256, 256)
    for i in range(2):
        ref, _ = oracle.msssim(xr[i].astype(float), yr[i].astype(float), L=1.0)
        assert abs(score[i].item() - ref) <= POOL_TOL


def test_msssim_identity_and_negative_domain(g, synth):
    x, _ = synth.luma_pairs_u8(1, 200, 200)
    xd = x.to(DEV)
    assert abs(g.msssim(xd, xd).item() - 1.0) <= 1e-7
    inv = (255 - x).to(DEV)
    s = g.msssim(xd, inv, scales=3, exponents=(0.3, 0.3, 0.4))
    ref, per = oracle.msssim(x[0].numpy(), (255 - x[0]).numpy(), scales=3, exponents=(0.3, 0.3, 0.4))
    assert np.isnan(ref) == np.isnan(s.item())


def test_msssim_1080p_batch_all_pairs(g, synth):
    """The benchmark's configuration (64 pairs of 1920x1080, the one
    persistent launch over all levels that bench.py times): every pair's
    score and every per-scale term (mean cs_j, mean Q_j) against the oracle."""
    n = 64
    x, y = synth.luma_pairs_u8(n, 1080, 1920, device=DEV)
    score, per = g.msssim(x, y, per_scale=True)
    xs, ys = x.cpu().numpy(), y.cpu().numpy()
    score, per = score.cpu().numpy(), per.cpu().numpy()
    for i in range(n):
        ref, ref_per = oracle.msssim(xs[i], ys[i])
        assert abs(score[i] - ref) <= POOL_TOL, (i, score[i], ref)
        np.testing.assert_allclose(per[i], np.array(ref_per), rtol=0, atol=POOL_TOL)
    assert (score > 0.5).all() and (score < 1).all()


def test_8k_pair_full_map_and_msssim(g, synth):
    """The largest frame size in the paper's workloads' range (7680 x 4320
    UHD-2): every element of the SSIM map, the pooled score and MS-SSIM
    against the oracle."""
    x, y = synth.single_pair_u8(4320, 7680)
    xd, yd = x.to(DEV), y.to(DEV)
    mean, q = g.ssim(xd, yd, return_map=True)
    ref_mean, ref = oracle.ssim(x.numpy(), y.numpy())
    _check_map(q[0].cpu().numpy(), ref["q"])
    assert abs(mean[0].item() - ref_mean) <= POOL_TOL
    s = g.msssim(xd, yd)
    ref_ms, _ = oracle.msssim(x.numpy(), y.numpy())
    assert abs(s[0].item() - ref_ms) <= POOL_TOL


def test_host_tensors_end_to_end(g, synth):
    x, y = synth.luma_pairs_u8(2, 180, 190)
    s_host = g.msssim(x, y)          # CPU tensors in, CPU result out
    s_dev = g.msssim(x.to(DEV), y.to(DEV)).cpu()
    assert s_host.device.type == "cpu" and torch.equal(s_host, s_dev)


def test_errors_reported(g):
    x = torch.zeros((1, 10, 40), dtype=torch.uint8, device=DEV)
    with pytest.raises(g.GbssimError) as e:
        g.ssim(x, x)
    assert e.value.status == g.ERR_TOO_SMALL
    x = torch.zeros((1, 100, 100), dtype=torch.uint8, device=DEV)
    with pytest.raises(g.GbssimError) as e:
        g.msssim(x, x)
    assert e.value.status == g.ERR_TOO_SMALL
