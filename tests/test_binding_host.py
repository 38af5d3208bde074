"""The Python binding's host-side logic on a CPU-only host: its constants
match the C header, parameter structs and plane descriptors are marshalled
as the header lays them out, and calls given host tensors where the C path
needs device memory refuse them (there is no CPU fallback)."""
import os
import re

import pytest
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def g():
    from paper_2101_06354_gb300 import build

    build.build()
    from paper_2101_06354_gb300 import gbssim

    return gbssim


def header_constants():
    src = open(os.path.join(ROOT, "include", "gbssim.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    out = {}
    for name, val in re.findall(r"^#define GBSSIM_([A-Z0-9_]+) +(\(?[-0-9 <()]+\)?)\s*$", src, flags=re.M):
        out[name] = eval(val)
    for name, val in re.findall(r"\bGBSSIM_([A-Z0-9_]+) = (-?[0-9]+)", src):
        out[name] = int(val)
    return out


def test_binding_constants_match_the_header(g):
    hdr = header_constants()
    shared = [n for n in hdr if hasattr(g, n)]
    assert len(shared) >= 45, shared  # status codes, dtypes, windows, ops, pool kinds, flags, limits
    for n in shared:
        assert getattr(g, n) == hdr[n], n
    assert g.DOWNSCALE_RULES == {"round_min": hdr["DOWNSCALE_ROUND_MIN"], "ceil_h": hdr["DOWNSCALE_CEIL_H"]}
    assert {k: v for k, v in g.POOL_KINDS.items()} == {n[5:].lower(): hdr[n] for n in hdr if n.startswith("POOL_")}


def test_make_params_marshalling(g):
    p = g.make_params(window="box", k=8, stride=4, L=1.0, scales=3, exponents=(0.2, 0.3, 0.5), combine="sum",
                      border="reflect", flags=g.FLAG_PYRAMID_97)
    assert (p.window, p.k, p.stride, p.scales, p.L) == (g.WIN_BOX, 8, 4, 3, 1.0)
    assert list(p.exponents) == [0.2, 0.3, 0.5] + [0.0] * (g.MAX_SCALES - 3)
    assert p.combine == g.COMBINE_SUM and p.flags == g.FLAG_BORDER_REFLECT | g.FLAG_PYRAMID_97
    d = g.make_params()
    assert (d.window, d.k, d.sigma, d.K1, d.K2, d.L, d.stride, d.scales) == (g.WIN_GAUSSIAN, 11, 1.5, 0.01, 0.03,
                                                                            255.0, 1, 5)
    with pytest.raises(ValueError):
        g.make_params(scales=3, exponents=(0.5, 0.5))
    with pytest.raises(KeyError):
        g.make_params(border="wrap")


def test_map_shapes(g):
    assert g.map_shape(1080, 1920, g.make_params()) == (1070, 1910)
    assert g.map_shape(1080, 1920, g.make_params(border="zero")) == (1080, 1920)
    assert g.map_shape(1080, 1920, g.make_params(border="reflect", k=8, window="box")) == (1080, 1920)
    assert g.map_shape(100, 101, g.make_params(window="box", k=8, stride=4)) == (24, 24)
    assert g.out_shape(11, 11, 11, 1) == (1, 1) and g.out_shape(10, 30, 11, 1)[0] == 0


def test_batch_views_and_plane_descriptors(g):
    t = torch.zeros(2, 3, 16, 24, dtype=torch.uint8)
    b = g._as_batch(t)
    assert b.shape == (6, 16, 24)
    pl = g.plane(b)
    assert (pl.dtype, pl.count, pl.height, pl.width, pl.row_stride, pl.image_stride) == (g.U8, 6, 16, 24, 24, 384)
    one = g.plane(g._as_batch(torch.zeros(16, 24, dtype=torch.float32)))
    assert (one.dtype, one.count, one.image_stride) == (g.F32, 1, 16 * 24)
    # a column window of wider rows keeps its row pitch (no copy)
    w = torch.zeros(4, 16, 40, dtype=torch.float16)[:, :, 8:32]
    pw = g.plane(g._as_batch(w))
    assert (pw.dtype, pw.width, pw.row_stride, pw.image_stride) == (g.F16, 24, 40, 640)
    assert pw.data == w.data_ptr()
    assert g.plane(g._as_batch(torch.zeros(3, 8, 8, dtype=torch.bfloat16))).dtype == g.BF16
    with pytest.raises(ValueError):
        g._as_batch(torch.zeros(16))
    with pytest.raises(TypeError):
        g.plane(torch.zeros(1, 8, 8, dtype=torch.float64))


def test_host_tensors_are_refused_not_computed(g):
    x = torch.zeros(1, 32, 32)
    with pytest.raises(ValueError):
        g.downscale(x, 2)  # block means run on the GPU only
    with pytest.raises(ValueError):
        g.msssim_host(x, torch.zeros(1, 32, 32, dtype=torch.uint8))  # mismatched pair, refused before any copy
    with pytest.raises(ValueError):
        g.ssim3d(torch.zeros(5, 32, 32), torch.zeros(5, 32, 32))  # SSIM-3D takes uint8 videos
