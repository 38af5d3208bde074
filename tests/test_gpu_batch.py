"""GPU tests of the ragged persistent batch (gbssim_batch_*), its CUDA-graph
replay, the bounded dependency wait, and the autotuner."""
import os

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


SIZES = [(360, 640), (480, 854), (720, 1280), (177, 203), (1013, 777), (401, 333), (360, 640), (199, 1001)]


def _pairs(synth, sizes, dtype=torch.uint8):
    xs, ys = synth.ragged_pairs_u8(sizes)
    if dtype != torch.uint8:
        xs = [x.to(dtype) / 255 for x in xs]
        ys = [y.to(dtype) / 255 for y in ys]
    return [x.to(DEV) for x in xs], [y.to(DEV) for y in ys]


@pytest.mark.parametrize("multiscale", [False, True])
def test_batch_matches_single_calls_and_oracle(g, synth, multiscale):
    xs, ys = _pairs(synth, SIZES)
    plan = g.BatchPlan(xs, ys, multiscale=multiscale)
    scores = plan.run().clone()
    torch.cuda.synchronize()
    assert plan.status() == 0
    for i, (x, y) in enumerate(zip(xs, ys)):
        single = (g.msssim if multiscale else g.ssim)(x, y)
        assert abs(scores[i].item() - single.item()) <= 1e-7  # fp32 pooling grouped by different segments
    for i in (0, 4, 7):
        if multiscale:
            ref, _ = oracle.msssim(xs[i].cpu().numpy(), ys[i].cpu().numpy())
        else:
            ref, _ = oracle.ssim(xs[i].cpu().numpy(), ys[i].cpu().numpy())
        assert abs(scores[i].item() - ref) <= 1e-6


def test_batch_float_inputs_and_multi_image_entries(g, synth):
    x, y = synth.loss_pairs_float(2, 2, 130, 150)
    xs = [x.reshape(4, 130, 150).to(DEV), x[0, 0, :100, :120].contiguous().to(DEV)]
    ys = [y.reshape(4, 130, 150).to(DEV), y[0, 0, :100, :120].contiguous().to(DEV)]
    plan = g.BatchPlan(xs, ys, L=1.0)
    scores = plan.run()
    ref = torch.cat([g.ssim(xs[0], ys[0], L=1.0), g.ssim(xs[1], ys[1], L=1.0)])
    assert torch.allclose(scores, ref, rtol=0, atol=1e-7)


@pytest.mark.parametrize("multiscale", [False, True])
def test_batch_deterministic_and_graph_replay(g, synth, multiscale):
    xs, ys = _pairs(synth, SIZES)
    plan = g.BatchPlan(xs, ys, multiscale=multiscale, seg_rows=64)
    a = plan.run().clone()
    b = plan.run().clone()
    assert torch.equal(a, b)  # fixed pooling slots: bit-identical whichever CTA ran which item
    plan.capture()
    plan.scores.zero_()
    r = plan.replay().clone()
    torch.cuda.synchronize()
    assert torch.equal(a, r)
    # refill the bound inputs in place: the replay scores the new data
    for y in ys:
        y.copy_(torch.flip(y, dims=[1]))
    r2 = plan.replay().clone()
    torch.cuda.synchronize()
    eager = torch.stack([(g.msssim if multiscale else g.ssim)(x, y)[0] for x, y in zip(xs, ys)])
    assert torch.allclose(r2, eager, rtol=0, atol=1e-7)
    assert not torch.equal(r2, a)


def test_batch_tuning_knobs_agree(g, synth):
    xs, ys = _pairs(synth, SIZES[:5])
    ref = g.BatchPlan(xs, ys, multiscale=True).run().clone()
    for rows, ctas in [(16, 1), (64, 2), (512, 0), (4096, 3)]:
        plan = g.BatchPlan(xs, ys, multiscale=True, seg_rows=rows, ctas_per_sm=ctas)
        assert torch.allclose(plan.run(), ref, rtol=0, atol=1e-7)


@pytest.mark.parametrize("tile_w", [32, 128])
@pytest.mark.parametrize("multiscale", [False, True])
def test_batch_strip_widths_agree(g, synth, tile_w, multiscale):
    """Strips of 32 and 128 output columns (128- and 512-thread CTAs) score as
    the 64-column default, and as the oracle; the odd sizes leave ragged last
    strips at every width."""
    xs, ys = _pairs(synth, SIZES)
    ref = g.BatchPlan(xs, ys, multiscale=multiscale).run().clone()
    plan = g.BatchPlan(xs, ys, multiscale=multiscale, tile_w=tile_w, seg_rows=128)
    got = plan.run().clone()
    torch.cuda.synchronize()
    assert plan.status() == 0
    assert torch.allclose(got, ref, rtol=0, atol=1e-7)
    for i in (3, 5):
        if multiscale:
            want, _ = oracle.msssim(xs[i].cpu().numpy(), ys[i].cpu().numpy())
        else:
            want, _ = oracle.ssim(xs[i].cpu().numpy(), ys[i].cpu().numpy())
        assert abs(got[i].item() - want) <= 1e-6
    fx, fy = _pairs(synth, SIZES[:3], dtype=torch.float32)
    fref = g.BatchPlan(fx, fy, multiscale=multiscale, L=1.0).run().clone()
    fgot = g.BatchPlan(fx, fy, multiscale=multiscale, L=1.0, tile_w=tile_w).run()
    assert torch.allclose(fgot, fref, rtol=0, atol=1e-7)


def test_bounded_wait_reports_timeout(g, synth):
    """The test hook makes image 0's level-1 items wait for a level-0 item that
    does not exist: the wait gives up after `wait_limit` spins, the kernel
    records GBSSIM_ERR_TIMEOUT and the launch still ends."""
    xs, ys = _pairs(synth, SIZES[:3])
    plan = g.BatchPlan(xs, ys, multiscale=True, wait_limit=2000, flags=g.TUNING_TEST_STALL)
    plan.run()
    torch.cuda.synchronize()
    assert plan.status() == g.ERR_TIMEOUT
    ok = g.BatchPlan(xs, ys, multiscale=True)
    ok.run()
    assert ok.status() == 0


def test_autotuner_picks_and_caches(g, synth, tmp_path, monkeypatch):
    from paper_2101_06354_gb300 import tune

    monkeypatch.setenv("GBSSIM_TUNE_CACHE", str(tmp_path / "tune.json"))
    xs, ys = _pairs(synth, SIZES[:4])
    rows, ctas, tw, res = tune.tune(xs, ys, multiscale=True,
                                    candidates=[(64, 0, 32), (256, 0), (128, 2, 64), (256, 0, 128)], reps=2)
    assert "%d/%d/%d" % (rows, ctas, tw) in res and len(res) == 4
    assert os.path.exists(tmp_path / "tune.json")
    rows2, ctas2, tw2, _ = tune.tune(xs, ys, multiscale=True, candidates=[(16, 1)], reps=1)
    assert (rows2, ctas2, tw2) == (rows, ctas, tw)   # served from the cache
    plan = tune.autotuned_plan(xs, ys, multiscale=True)
    assert plan.seg_rows == rows and plan.tile_w == tw
    ref = g.BatchPlan(xs, ys, multiscale=True).run()
    assert torch.allclose(plan.run(), ref, rtol=0, atol=1e-7)
