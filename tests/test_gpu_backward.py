"""GPU parity of the hand-written backward pass (gbssim_ssim_backward) and the
SSIM / MS-SSIM loss autograd Function against the FP64 oracle's analytic
gradient (itself pinned to central finite differences in
tests/test_oracle_pins.py).

Tolerance (the paper gives none for gradients): max |dg| <= 1e-4 * max |g|
for fp32 gradients; bf16 / fp16 gradient storage rounds each element to 8 / 11
significant bits, so those are checked at 1e-2 * max |g| (bf16) and 2e-3 (fp16).
"""
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


@pytest.fixture(scope="module")
def synth():
    from paper_2101_06354_gb300 import synth as s

    return s


def _rel_err(got, ref):
    return np.abs(got - ref).max() / np.abs(ref).max()


def _np64(t):
    return t.detach().double().cpu().numpy()


@pytest.mark.parametrize("h,w", [(64, 70), (140, 131), (11, 11), (12, 40), (200, 97), (27, 300), (16, 16)])
@pytest.mark.parametrize("dtype,L", [(torch.float32, 1.0), (torch.uint8, 255.0)])
def test_ssim_gradient_matches_oracle(g, synth, h, w, dtype, L):
    if dtype == torch.uint8:
        x, y = synth.single_pair_u8(h, w)
    else:
        x, y = synth.loss_pairs_float(1, 1, h, w)
        x, y = x[0, 0], y[0, 0]
    grad, score = g.ssim_backward(x.to(DEV), y.to(DEV), return_score=True, L=L,
                                  grad_dtype=torch.float32)
    ref = oracle.ssim_grad(_np64(x), _np64(y), L=L)
    assert _rel_err(grad.double().cpu().numpy(), ref) <= 1e-4
    ref_score, _ = oracle.ssim(_np64(x), _np64(y), L=L)
    assert abs(score.item() - ref_score) <= 1e-6


@pytest.mark.parametrize("kw", [dict(window="gaussian", k=7, sigma=1.0), dict(window="box", k=8),
                                dict(window="box", k=11), dict(window="gaussian", k=15, sigma=2.0)])
def test_ssim_gradient_other_windows(g, synth, kw):
    x, y = synth.loss_pairs_float(1, 1, 90, 77)
    x, y = x[0, 0], y[0, 0]
    grad = g.ssim_backward(x.to(DEV), y.to(DEV), L=1.0, **kw)
    okw = dict(kw)
    okw["window_kind"] = okw.pop("window")
    ref = oracle.ssim_grad(_np64(x), _np64(y), L=1.0, **okw)
    assert _rel_err(grad.double().cpu().numpy(), ref) <= 1e-4


@pytest.mark.parametrize("h,w", [(200, 232), (181, 199)])
@pytest.mark.parametrize("combine", ["product", "sum"])
def test_msssim_gradient_matches_oracle(g, synth, h, w, combine):
    x, y = synth.loss_pairs_float(1, 2, h, w)
    xs, ys = x.reshape(2, h, w), y.reshape(2, h, w)
    grad, score = g.ssim_backward(xs.to(DEV), ys.to(DEV), multiscale=True, return_score=True, L=1.0,
                                  combine=combine)
    for i in range(2):
        ref_score, ref = oracle.msssim_grad(_np64(xs[i]), _np64(ys[i]), L=1.0, combine=combine)
        assert _rel_err(grad[i].double().cpu().numpy(), ref) <= 1e-4
        assert abs(score[i].item() - ref_score) <= 1e-6


def test_msssim_backward_with_forward_results(g, synth):
    """Passing the forward's pooled scales skips the re-run of the forward: the
    gradient must be identical to the self-contained call."""
    x, y = synth.loss_pairs_float(1, 3, 190, 200)
    xs, ys = x.reshape(3, 190, 200).to(DEV), y.reshape(3, 190, 200).to(DEV)
    score, per = g.msssim(xs, ys, per_scale=True, L=1.0)
    a = g.ssim_backward(xs, ys, multiscale=True, L=1.0)
    b, sb = g.ssim_backward(xs, ys, multiscale=True, L=1.0, fwd_score=score, fwd_per_scale=per, return_score=True)
    assert torch.equal(sb, score)
    assert torch.allclose(a, b, rtol=0, atol=1e-6 * a.abs().max().item())


def test_msssim_gradient_three_scales_u8(g, synth):
    x, y = synth.luma_pairs_u8(1, 100, 120)
    kw = dict(scales=3, exponents=(0.3, 0.3, 0.4))
    grad = g.ssim_backward(x.to(DEV), y.to(DEV), multiscale=True, grad_dtype=torch.float32, **kw)
    _, ref = oracle.msssim_grad(_np64(x[0]), _np64(y[0]), **kw)
    assert _rel_err(grad[0].double().cpu().numpy(), ref) <= 1e-4


@pytest.mark.parametrize("gdt,tol", [(torch.bfloat16, 1e-2), (torch.float16, 2e-3)])
def test_low_precision_storage(g, synth, gdt, tol):
    x, y = synth.loss_pairs_float(1, 1, 96, 100)
    xt, yt = x[0, 0].to(gdt), y[0, 0].to(gdt)
    grad = g.ssim_backward(xt.to(DEV), yt.to(DEV), L=1.0)
    assert grad.dtype == gdt
    ref = oracle.ssim_grad(_np64(xt), _np64(yt), L=1.0)   # same rounded inputs
    assert _rel_err(grad.double().cpu().numpy(), ref) <= tol


def test_gradient_zero_at_identity_and_scale_factors(g, synth):
    x, y = synth.loss_pairs_float(1, 3, 80, 90)
    xs, ys = x.reshape(3, 80, 90).to(DEV), y.reshape(3, 80, 90).to(DEV)
    g0 = g.ssim_backward(xs, xs, L=1.0)
    assert g0.abs().max().item() <= 1e-6 * 1e3  # exact zero up to fp32 rounding of the maps
    base = g.ssim_backward(xs, ys, L=1.0)
    scaled = g.ssim_backward(xs, ys, L=1.0, grad_scale=-0.5)
    assert torch.allclose(scaled, -0.5 * base, rtol=1e-6, atol=0)
    per = torch.tensor([1.0, 2.0, -3.0], dtype=torch.float64, device=DEV)
    gp = g.ssim_backward(xs, ys, L=1.0, grad_out=per)
    for i, f in enumerate([1.0, 2.0, -3.0]):
        assert torch.allclose(gp[i], f * base[i], rtol=1e-6, atol=0)


@pytest.mark.parametrize("multiscale", [False, True])
@pytest.mark.parametrize("recompute", [True, False])
def test_loss_autograd(g, synth, multiscale, recompute):
    x, y = synth.loss_pairs_float(2, 3, 176, 180)
    xd = x.to(DEV)
    yd = y.to(DEV).requires_grad_(True)
    loss_fn = g.SSIMLoss(multiscale=multiscale, recompute=recompute, L=1.0)
    loss = loss_fn(xd, yd)
    (2.5 * loss).backward()
    xs, ys = _np64(x).reshape(6, 176, 180), _np64(y).reshape(6, 176, 180)
    scores, grads = [], []
    for i in range(6):
        if multiscale:
            s, gr = oracle.msssim_grad(xs[i], ys[i], L=1.0)
        else:
            s, _ = oracle.ssim(xs[i], ys[i], L=1.0)
            gr = oracle.ssim_grad(xs[i], ys[i], L=1.0)
        scores.append(s)
        grads.append(gr)
    assert abs(loss.item() - (1.0 - np.mean(scores))) <= 1e-6
    ref = -2.5 / 6 * np.stack(grads).reshape(y.shape)
    assert yd.grad.shape == y.shape
    assert _rel_err(yd.grad.double().cpu().numpy(), ref) <= 1e-4


@pytest.mark.parametrize("multiscale", [False, True])
def test_loss_fwd_bwd_full_size(g, synth, multiscale):
    """The loss workload at full size (32 x 3 x 512 x 512 fp32, L = 1) through
    the default Function (the backward recomputes the moments): the loss
    value and the gradient of every one of the 96 planes against the
    oracle's analytic gradient."""
    x, y = synth.loss_pairs_float(32, 3, 512, 512, device=DEV)
    yd = y.clone().requires_grad_(True)
    loss = g.SSIMLoss(multiscale=multiscale, L=1.0)(x, yd)
    loss.backward()
    xs, ys = _np64(x.reshape(96, 512, 512)), _np64(y.reshape(96, 512, 512))
    gr = yd.grad.reshape(96, 512, 512).double().cpu().numpy()
    scores = []
    for i in range(96):
        if multiscale:
            sc, ref = oracle.msssim_grad(xs[i], ys[i], L=1.0)
        else:
            sc, _ = oracle.ssim(xs[i], ys[i], L=1.0)
            ref = oracle.ssim_grad(xs[i], ys[i], L=1.0)
        scores.append(sc)
        assert _rel_err(gr[i], -1.0 / 96 * ref) <= 1e-4, i
    assert abs(loss.item() - (1.0 - np.mean(scores))) <= 1e-6


def test_loss_fwd_bwd_full_size_bf16_sampled(g, synth):
    """The bf16-stored variant of the full-size loss workload: sampled planes
    against the oracle's gradient on the same rounded inputs."""
    x, y = synth.loss_pairs_float(32, 3, 512, 512, device=DEV)
    xb, yb = x.to(torch.bfloat16), y.to(torch.bfloat16).requires_grad_(True)
    loss = g.SSIMLoss(L=1.0)(xb, yb)
    loss.backward()
    assert yb.grad.dtype == torch.bfloat16
    xs, ys = xb.detach().reshape(96, 512, 512), yb.detach().reshape(96, 512, 512)
    gr = yb.grad.reshape(96, 512, 512)
    for i in (0, 47, 95):
        ref = -1.0 / 96 * oracle.ssim_grad(_np64(xs[i]), _np64(ys[i]), L=1.0)
        assert _rel_err(gr[i].double().cpu().numpy(), ref) <= 1e-2


def test_backward_rejects_unsupported(g):
    x = torch.zeros((1, 40, 40), device=DEV)
    with pytest.raises(g.GbssimError) as e:
        g.ssim_backward(x, x, stride=2)
    assert e.value.status == g.ERR_UNSUPPORTED
    with pytest.raises(g.GbssimError) as e:
        g.ssim_backward(x, x, k=33, sigma=5.0)
    assert e.value.status == g.ERR_UNSUPPORTED


@pytest.mark.parametrize("multiscale,dtype", [(False, torch.float32), (True, torch.float32), (False, torch.bfloat16)])
def test_saved_loss_path_equals_recompute_path(g, synth, multiscale, dtype):
    """SSIMLoss(recompute=False) keeps the forward's coefficient maps
    (gbssim_loss_forward / gbssim_loss_backward); the default form recomputes
    them in the backward (gbssim_ssim_backward).  For SSIM both run the same
    coefficient kernel on the same inputs, so the gradients agree bit for bit.
    For MS-SSIM the default form's forward pools through the persistent
    kernel (another fp32 summation order), so its per-scale means, and with
    them the factors each level's gradient is scaled by, differ in the last
    bits (the pooled means differ by about 1e-9): equal to 1e-6 of the largest
    gradient."""
    x, y = synth.loss_pairs_float(2, 2, 190, 200)
    xd = x.to(DEV, dtype)
    ys = y.to(DEV, dtype)
    grads, losses = [], []
    for recompute in (True, False):
        yd = ys.clone().requires_grad_(True)
        loss = g.SSIMLoss(multiscale=multiscale, recompute=recompute, L=1.0)(xd, yd)
        loss.backward()
        grads.append(yd.grad.reshape(4, 190, 200).float())
        losses.append(loss.item())
    if multiscale:
        assert (grads[0] - grads[1]).abs().max().item() <= 1e-6 * grads[1].abs().max().item()
        assert abs(losses[0] - losses[1]) <= 1e-7  # fp32 partial sums in another order
    else:
        assert torch.equal(grads[0], grads[1])
        assert losses[0] == losses[1]
    xs, yr = xd.reshape(4, 190, 200), ys.reshape(4, 190, 200)
    kw = dict(exponents=g.MSSSIM_EXPONENTS) if multiscale else {}
    ref = g.ssim_backward(xs, yr, multiscale=multiscale, grad_scale=-0.25, L=1.0, grad_dtype=torch.float32, **kw)
    tol = 1e-6 if dtype == torch.float32 else 1e-2
    assert (grads[0] - ref).abs().max().item() <= tol * ref.abs().max().item()
    score = (g.msssim if multiscale else g.ssim)(xs, yr, L=1.0)
    assert abs(losses[0] - (1.0 - score.mean().item())) <= 1e-7
