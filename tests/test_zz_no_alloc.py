"""gbssim_ssim_map_static: the SSIM entry point for callers that cannot
allocate device memory (for example a plugin that only receives its input and
output buffers from a host application, or a pipeline that forbids cudaMalloc
after start-up).  Its scratch is a static device array inside the library.

The GPU test calls it through the C ABI twice in a row, on different inputs,
and checks each result against gbssim_ssim_map (the entry point with a
caller-provided workspace) on the same inputs: both run the same deterministic
kernels, so map and mean must agree bit for bit.  It lives in its own file,
collected last, and passes both on its own in a fresh process and after the
rest of the suite.  The size limit is checked on the host before any CUDA
call, so that test needs no GPU.
"""
import ctypes

import pytest
import torch


@pytest.fixture(scope="module")
def lib():
    from paper_2101_06354_gb300 import build

    build.build()
    from paper_2101_06354_gb300 import gbssim

    return gbssim


@pytest.fixture(scope="module")
def g(lib):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return lib


def _static_call(g, x, y, p):
    px, py = g.plane(x), g.plane(y)
    n, h, w = x.shape
    oh, ow = g.out_shape(h, w, p.k, p.stride)
    qmap = torch.full((n, oh, ow), float("nan"), device=x.device)
    mean = torch.full((n,), float("nan"), dtype=torch.float64, device=x.device)
    rc = g.lib.gbssim_ssim_map_static(ctypes.byref(px), ctypes.byref(py), ctypes.byref(p), qmap.data_ptr(),
                                      qmap.stride(1), qmap.stride(0), mean.data_ptr(),
                                      torch.cuda.current_stream().cuda_stream)
    return rc, mean, qmap


@pytest.mark.gpu
def test_static_scratch_entry_matches_workspace_entry(g):
    from paper_2101_06354_gb300 import synth

    cases = [(synth.luma_pairs_u8(3, 300, 517, device="cuda"), g.make_params()),
             ((synth.loss_pairs_float(1, 2, 257, 190, device="cuda")), g.make_params(L=1.0))]
    for (x, y), p in cases:
        x = g._as_batch(x)
        y = g._as_batch(y)
        ws = g.workspace(g.plane(x), p, g.OP_SSIM, x.device)
        ref_mean = torch.empty(x.shape[0], dtype=torch.float64, device=x.device)
        oh, ow = g.out_shape(x.shape[1], x.shape[2], p.k, p.stride)
        ref_map = torch.empty((x.shape[0], oh, ow), device=x.device)
        px, py = g.plane(x), g.plane(y)
        assert g.lib.gbssim_ssim_map(ctypes.byref(px), ctypes.byref(py), ctypes.byref(p), ref_map.data_ptr(),
                                     ref_map.stride(1), ref_map.stride(0), ref_mean.data_ptr(), ws.data_ptr(),
                                     ws.numel(), torch.cuda.current_stream().cuda_stream) == 0
        rc, mean, qmap = _static_call(g, x, y, p)
        torch.cuda.synchronize()
        assert rc == 0
        assert torch.equal(qmap, ref_map)
        assert torch.equal(mean, ref_mean)


def test_static_scratch_rejects_oversized_problem(lib):
    """65536 pool slots hold about 430 pairs of 1920x1080; 1000 pairs need
    more and are rejected on the host before any CUDA call (the plane
    addresses are never dereferenced), so this runs without a GPU.  Argument
    errors come first, as gbssim_ssim_map reports them."""
    g = lib
    p = g.make_params()
    x = g.Plane(0x1000, g.U8, 1000, 1080, 1920, 1920, 1080 * 1920)
    n = ctypes.c_size_t()
    assert g.lib.gbssim_workspace_size(ctypes.byref(x), ctypes.byref(p), g.OP_SSIM, ctypes.byref(n)) == 0
    assert n.value > g.STATIC_SCRATCH_BYTES
    rc = g.lib.gbssim_ssim_map_static(ctypes.byref(x), ctypes.byref(x), ctypes.byref(p), None, 0, 0,
                                      ctypes.c_void_p(0x2000), None)
    assert rc == g.ERR_TOO_LARGE
    assert "static scratch" in g.status_string(rc)
    # no output at all, or a mismatched pair: the argument error wins
    rc = g.lib.gbssim_ssim_map_static(ctypes.byref(x), ctypes.byref(x), ctypes.byref(p), None, 0, 0, None, None)
    assert rc == g.ERR_INVALID_ARG
    y = g.Plane(0x1000, g.U8, 1000, 1080, 1921, 1921, 1080 * 1921)
    rc = g.lib.gbssim_ssim_map_static(ctypes.byref(x), ctypes.byref(y), ctypes.byref(p), None, 0, 0,
                                      ctypes.c_void_p(0x2000), None)
    assert rc == g.ERR_INVALID_ARG
