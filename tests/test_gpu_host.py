"""gbssim_msssim_host: MS-SSIM of host-resident pairs with the host-to-device
copies overlapped with compute.  Chunked mode runs gbssim_msssim's
computation; each pair's score depends only on its own work items, so
chunking must not change a single bit of it.  Streamed mode (chunks = 0)
cuts the two largest levels into shorter work items (another fp32 summation
order), so it is held to the oracle at the pooled parity bound instead."""
import ctypes
import os
import subprocess
import sys

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


@pytest.mark.parametrize("n,h,w,chunks", [(7, 200, 232, 3), (5, 181, 203, 1), (6, 256, 320, 6), (1, 200, 240, 4),
                                          (9, 184, 200, 8)])
def test_host_pipeline_equals_device_call(g, synth, n, h, w, chunks):
    x, y = synth.luma_pairs_u8(n, h, w)
    ref = g.msssim(x.to(DEV), y.to(DEV)).cpu()
    got = g.msssim_host(x.pin_memory(), y.pin_memory(), chunks=chunks)
    assert got.shape == (n,)
    assert torch.equal(got, ref)
    one = g.msssim_host(x.pin_memory(), y.pin_memory(), chunks=chunks, two_compute_streams=False)
    assert torch.equal(one, ref)
    s0, _ = oracle.msssim(x[0].numpy(), y[0].numpy())
    assert abs(got[0].item() - s0) <= 1e-6


# (n, h, w): several 128-row level-0 items with a ragged last one (600 rows),
# one image, a group per image (n <= 16) and uneven groups of several images (n = 37)
@pytest.mark.parametrize("n,h,w", [(7, 200, 232), (5, 181, 203), (1, 200, 240), (3, 600, 300), (37, 176, 176)])
def test_streamed_matches_oracle(g, synth, n, h, w):
    x, y = synth.luma_pairs_u8(n, h, w)
    got = g.msssim_host(x.pin_memory(), y.pin_memory(), chunks=0)
    assert got.shape == (n,)
    dev = g.msssim(x.to(DEV), y.to(DEV)).cpu()
    assert torch.allclose(got, dev, rtol=0, atol=1e-6)
    for i in range(n):
        s, _ = oracle.msssim(x[i].numpy(), y[i].numpy())
        assert abs(got[i].item() - s) <= 1e-6
    # a second call on the same buffers (flags cleared per call)
    assert torch.equal(g.msssim_host(x.pin_memory(), y.pin_memory(), chunks=0), got)


def test_streamed_full_size_all_pairs(g, synth):
    """The end-to-end benchmark step: 64 pinned 1920x1080 pairs streamed
    through one launch (eight copy groups of 6 pairs, then groups of 4, 4, 2,
    2, 1, 1, 1, 1; 128-row items at the two largest levels); every score
    against the device call and against the oracle."""
    n = 64
    x, y = synth.luma_pairs_u8(n, 1080, 1920)
    got = g.msssim_host(x.pin_memory(), y.pin_memory(), chunks=0)
    dev = g.msssim(x.to(DEV), y.to(DEV)).cpu()
    assert torch.isfinite(got).all()
    assert torch.allclose(got, dev, rtol=0, atol=1e-6)
    xs, ys = x.numpy(), y.numpy()
    for i in range(n):
        s, _ = oracle.msssim(xs[i], ys[i])
        assert abs(got[i].item() - s) <= 1e-6, (i, got[i].item(), s)


def test_streamed_arrival_wait_reports_timeout(g, synth):
    """The test hook leaves the last copy group's arrival flag unset: the
    level-0 items of its image wait until their bounded wait (16 x wait_limit
    polls) runs out, the launch records GBSSIM_ERR_TIMEOUT, that image scores
    NaN, and the call still completes.  37 pairs make eight copy groups of 2
    or 3 images and then groups of 4, 4, 2, 2, 1, 1, 1, 1: the last holds one
    image."""
    n = 37
    x, y = synth.luma_pairs_u8(n, 176, 176)
    xp, yp = x.pin_memory(), y.pin_memory()
    dev = g.msssim(x.to(DEV), y.to(DEV)).cpu()
    status = torch.full((1,), 12345, dtype=torch.int32).pin_memory()
    t = g.Tuning(0, 0, 4000, g.TUNING_TEST_DROP_ARRIVAL)
    got = g.msssim_host(xp, yp, chunks=0, tuning=t, status=status)
    assert status.item() == g.ERR_TIMEOUT
    assert torch.isnan(got[n - 1])
    fin = torch.isfinite(got)
    assert torch.allclose(got[fin], dev[fin], rtol=0, atol=1e-6)
    # the same buffers again without the hook: every flag set, status OK
    status.fill_(12345)
    got = g.msssim_host(xp, yp, chunks=0, tuning=g.Tuning(0, 0, 0, 0), status=status)
    assert status.item() == 0
    assert torch.allclose(got, dev, rtol=0, atol=1e-6)
    # the status word and the hook belong to streamed mode
    with pytest.raises(g.GbssimError) as e:
        g.msssim_host(xp, yp, chunks=2, status=status)
    assert e.value.status == g.ERR_UNSUPPORTED


_BLOCKING_SCRIPT = """
import torch
from paper_2101_06354_gb300 import gbssim, synth
x, y = synth.luma_pairs_u8(20, 176, 176)
dev = gbssim.msssim(x.cuda(), y.cuda()).cpu()
got = gbssim.msssim_host(x.pin_memory(), y.pin_memory(), chunks=0)
assert torch.isfinite(got).all(), got
assert torch.allclose(got, dev, rtol=0, atol=1e-6), (got - dev).abs().max()
print("streamed ok")
"""


def test_streamed_with_blocking_launches(g):
    """With every kernel launch blocking the host, the streamed launch must
    still find its inputs arriving: all copies are enqueued before it."""
    env = dict(os.environ, CUDA_LAUNCH_BLOCKING="1")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", _BLOCKING_SCRIPT], env=env, cwd=root, capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0 and "streamed ok" in r.stdout, r.stdout + r.stderr


def test_host_pipeline_strided_and_pageable(g, synth):
    x, y = synth.luma_pairs_u8(4, 200, 240)
    xs, ys = x[:, :, 8:232], y[:, :, 8:232]  # row pitch 240 > width 224: per-image 2-D copies
    ref = g.msssim(xs.contiguous().to(DEV), ys.contiguous().to(DEV)).cpu()
    assert torch.equal(g.msssim_host(xs, ys, chunks=2), ref)  # pageable memory: correct, not overlapped
    assert torch.allclose(g.msssim_host(xs, ys, chunks=0), ref, rtol=0, atol=1e-6)  # streamed, pageable
    # the public call routes host tensors through the pipeline
    assert torch.equal(g.msssim(xs.contiguous().pin_memory(), ys.contiguous().pin_memory()), ref)


def test_host_pipeline_float_and_scales(g, synth):
    x, y = synth.loss_pairs_float(2, 2, 150, 170)
    xs, ys = x.reshape(4, 150, 170), y.reshape(4, 150, 170)
    kw = dict(L=1.0, scales=3, exponents=(0.3, 0.3, 0.4))
    ref = g.msssim(xs.to(DEV), ys.to(DEV), **kw).cpu()
    assert torch.equal(g.msssim_host(xs.pin_memory(), ys.pin_memory(), chunks=3, **kw), ref)
    got = g.msssim_host(xs.pin_memory(), ys.pin_memory(), chunks=0, **kw)
    for i in range(4):
        s, _ = oracle.msssim(xs[i].double().numpy(), ys[i].double().numpy(), **kw)
        assert abs(got[i].item() - s) <= 1e-6


def test_host_pipeline_rejects_one_stream(g, synth):
    x, y = synth.luma_pairs_u8(2, 64, 64)
    px, py = g.plane(x), g.plane(y)
    p = g.make_params(exponents=g.MSSSIM_EXPONENTS[:2], scales=2)
    nb = ctypes.c_size_t()
    assert g.lib.gbssim_msssim_host_workspace_size(ctypes.byref(px), ctypes.byref(p), 2, ctypes.byref(nb)) == 0
    ws = torch.empty(nb.value, dtype=torch.uint8, device=DEV)
    out = torch.empty(2, dtype=torch.float64).pin_memory()
    st = torch.cuda.current_stream().cuda_stream
    cs = g._copy_stream(torch.device(DEV)).cuda_stream
    rc = g.lib.gbssim_msssim_host(ctypes.byref(px), ctypes.byref(py), ctypes.byref(p), 2, out.data_ptr(),
                                  ws.data_ptr(), ws.numel(), st, st, None)
    assert rc == g.ERR_INVALID_ARG
    rc = g.lib.gbssim_msssim_host(ctypes.byref(px), ctypes.byref(py), ctypes.byref(p), 2, out.data_ptr(),
                                  ws.data_ptr(), ws.numel(), st, cs, cs)  # second compute stream = copy stream
    assert rc == g.ERR_INVALID_ARG
    rc = g.lib.gbssim_msssim_host(ctypes.byref(px), ctypes.byref(py), ctypes.byref(p), 2, out.data_ptr(),
                                  ws.data_ptr(), nb.value - 1, st, cs, None)
    assert rc == g.ERR_WORKSPACE


def test_streamed_mode_checks(g, synth):
    """Streamed mode (chunks = 0) needs the persistent path's parameters and a
    copy stream that never synchronises with the compute stream."""
    x, y = synth.luma_pairs_u8(2, 64, 64)
    px, py = g.plane(x), g.plane(y)
    p = g.make_params(exponents=g.MSSSIM_EXPONENTS[:2], scales=2)
    nb = ctypes.c_size_t()
    assert g.lib.gbssim_msssim_host_workspace_size(ctypes.byref(px), ctypes.byref(p), 0, ctypes.byref(nb)) == 0
    p7 = g.make_params(k=7, sigma=1.0, exponents=g.MSSSIM_EXPONENTS[:2], scales=2)
    assert g.lib.gbssim_msssim_host_workspace_size(ctypes.byref(px), ctypes.byref(p7), 0,
                                                   ctypes.byref(ctypes.c_size_t())) == g.ERR_UNSUPPORTED
    ws = torch.empty(nb.value, dtype=torch.uint8, device=DEV)
    out = torch.empty(2, dtype=torch.float64).pin_memory()
    st = g._copy_stream(torch.device(DEV), 1).cuda_stream  # a non-blocking compute stream
    # the legacy default stream as copy stream synchronises with every blocking stream: refused
    rc = g.lib.gbssim_msssim_host(ctypes.byref(px), ctypes.byref(py), ctypes.byref(p), 0, out.data_ptr(),
                                  ws.data_ptr(), ws.numel(), st, None, None)
    assert rc == g.ERR_INVALID_ARG
    torch.cuda.synchronize()
