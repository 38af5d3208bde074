"""Host-side checks of the C ABI (no GPU needed).

The library must load, export every function declared in include/gbssim.h,
and reject bad arguments on the host before anything reaches the GPU (these
calls return before any CUDA runtime call, so they run on a CPU-only host).
"""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def g():
    from paper_2101_06354_gb300 import build

    build.build()
    from paper_2101_06354_gb300 import gbssim

    return gbssim


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(gbssim_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


def test_every_declared_symbol_is_exported(g):
    names = declared_functions()
    assert "gbssim_ssim_map" in names and "gbssim_msssim" in names
    for n in names:
        assert hasattr(g.lib, n), n


def test_status_strings_and_version(g):
    assert g.lib.gbssim_version() == 1
    for s in range(-7, 1):
        assert g.status_string(s)
    assert g.status_string(-99) == "unknown status"


def test_defaults_follow_recommended_parameters(g):
    p = g.Params()
    g.lib.gbssim_params_default(ctypes.byref(p))
    assert (p.window, p.k, p.sigma, p.K1, p.K2, p.L, p.stride, p.scales) == (0, 11, 1.5, 0.01, 0.03, 255.0, 1, 5)
    assert list(p.exponents)[:5] == [0.0448, 0.2856, 0.3001, 0.2363, 0.1333]


def _plane(g, h=64, w=80, n=1, dtype=0, ptr=0x1000, rs=None, is_=None):
    rs = w if rs is None else rs
    return g.Plane(ptr, dtype, n, h, w, rs, h * rs if is_ is None else is_)


def _ws(g, x, p, op):
    n = ctypes.c_size_t()
    rc = g.lib.gbssim_workspace_size(ctypes.byref(x), ctypes.byref(p), op, ctypes.byref(n))
    return rc, n.value


def test_workspace_sizes(g):
    p = g.make_params()
    rc, n1 = _ws(g, _plane(g, 1080, 1920), p, g.OP_SSIM)
    assert rc == 0 and n1 > 0 and n1 % 256 == 0
    rc, n64 = _ws(g, _plane(g, 1080, 1920, 64), p, g.OP_SSIM)
    # one fp64 (sum Q, sum cs) pair per work item and image
    assert rc == 0 and n64 > n1 and n64 >= 64 * 16 * 30
    rc, m = _ws(g, _plane(g, 1080, 1920, 2), p, g.OP_MSSSIM)
    # pyramid levels 2..5 of two pairs, x and y, fp32
    pyr = sum((1080 >> j) * (1920 >> j) for j in range(1, 5)) * 2 * 2 * 4
    assert rc == 0 and m >= pyr
    assert _ws(g, _plane(g, 100, 100), p, g.OP_MSSSIM)[0] == g.ERR_TOO_SMALL  # 100 -> 50 -> 25 -> 12 -> 6 < 11
    assert _ws(g, _plane(g, 100, 100), g.make_params(scales=3), g.OP_MSSSIM)[0] == 0


@pytest.mark.parametrize("field,value,status", [
    ("k", 0, -1), ("k", 64, -1), ("stride", 0, -1), ("scales", 0, -1), ("scales", 9, -1),
    ("window", 7, -1), ("sigma", 0.0, -1), ("L", -1.0, -1), ("combine", 3, -1), ("flags", 16, -1), ("flags", 12, -1),
])
def test_bad_params_rejected(g, field, value, status):
    p = g.make_params()
    setattr(p, field, value)
    x = _plane(g)
    mean = ctypes.c_void_p(0x2000)
    rc = g.lib.gbssim_ssim_map(ctypes.byref(x), ctypes.byref(x), ctypes.byref(p), None, 0, 0, mean,
                               ctypes.c_void_p(0x3000), 1 << 20, None)
    assert rc == status


def test_bad_planes_rejected(g):
    p = g.make_params()
    ok = _plane(g)
    call = lambda a, b, ws=1 << 20: g.lib.gbssim_ssim_map(ctypes.byref(a), ctypes.byref(b), ctypes.byref(p),
                                                          None, 0, 0, ctypes.c_void_p(0x2000),
                                                          ctypes.c_void_p(0x3000), ws, None)
    assert call(_plane(g, ptr=0), ok) == g.ERR_INVALID_ARG          # null data
    assert call(ok, _plane(g, w=81)) == g.ERR_INVALID_ARG           # shape mismatch
    assert call(ok, _plane(g, dtype=3)) == g.ERR_INVALID_ARG        # dtype mismatch
    assert call(_plane(g, dtype=9), _plane(g, dtype=9)) == g.ERR_INVALID_ARG
    assert call(_plane(g, rs=10), _plane(g, rs=10)) == g.ERR_INVALID_ARG  # row stride < width
    assert call(_plane(g, h=10), _plane(g, h=10)) == g.ERR_TOO_SMALL  # k = 11 > H
    assert call(ok, ok, ws=16) == g.ERR_WORKSPACE
    x2 = _plane(g, n=2, is_=10)
    assert call(x2, x2) == g.ERR_INVALID_ARG                       # overlapping images
    # neither a map nor a mean requested
    assert g.lib.gbssim_ssim_map(ctypes.byref(ok), ctypes.byref(ok), ctypes.byref(p), None, 0, 0, None,
                                 ctypes.c_void_p(0x3000), 1 << 20, None) == g.ERR_INVALID_ARG


def test_msssim_and_window_sums_validation(g):
    p = g.make_params()
    x = _plane(g, 150, 150)
    ws = ctypes.c_void_p(0x3000)
    assert g.lib.gbssim_msssim(ctypes.byref(x), ctypes.byref(x), ctypes.byref(p), ctypes.c_void_p(0x10), None,
                               ws, 1 << 30, None) == g.ERR_TOO_SMALL   # 150 -> 9 at scale 5
    assert g.lib.gbssim_msssim(ctypes.byref(x), ctypes.byref(x), ctypes.byref(p), None, None,
                               ws, 1 << 30, None) == g.ERR_INVALID_ARG
    xf = _plane(g, dtype=3)
    assert g.lib.gbssim_window_sums(ctypes.byref(xf), ctypes.byref(xf), 8, 4, ctypes.c_void_p(0x10), None) \
        == g.ERR_UNSUPPORTED
    xu = _plane(g)
    assert g.lib.gbssim_window_sums(ctypes.byref(xu), ctypes.byref(xu), 0, 4, ctypes.c_void_p(0x10), None) \
        == g.ERR_INVALID_ARG
    assert g.lib.gbssim_window_sums(ctypes.byref(xu), ctypes.byref(xu), 65, 1, ctypes.c_void_p(0x10), None) \
        == g.ERR_INVALID_ARG


def test_pool_validation(g):
    m = ctypes.c_void_p(0x1000)
    assert g.lib.gbssim_ssim_pool(m, 10, 10, 5, 1, 0, 0, None, ctypes.c_void_p(0x10), ctypes.c_void_p(0x20),
                                  1 << 20, None) == g.ERR_INVALID_ARG  # ld < w
    assert g.lib.gbssim_ssim_pool(m, 10, 10, 10, 1, 0, 42, None, ctypes.c_void_p(0x10), ctypes.c_void_p(0x20),
                                  1 << 20, None) == g.ERR_INVALID_ARG  # unknown kind

    def pool(kind, args, ws_bytes=1 << 20):
        a = (ctypes.c_double * 2)(*args) if args is not None else None
        return g.lib.gbssim_ssim_pool(m, 10, 10, 10, 1, 0, kind, a, ctypes.c_void_p(0x10), ctypes.c_void_p(0x20),
                                      ws_bytes, None)

    assert pool(g.POOL_MINKOWSKI, None) == g.ERR_INVALID_ARG       # p missing
    assert pool(g.POOL_DW, (-1.0, 0.0)) == g.ERR_INVALID_ARG       # p < 0
    assert pool(g.POOL_MD, (0.0, 1.0)) == g.ERR_INVALID_ARG        # p must be > 0
    assert pool(g.POOL_PERCENTILE, (101.0, 0.0)) == g.ERR_INVALID_ARG
    assert pool(g.POOL_PP, (10.0, 0.0)) == g.ERR_INVALID_ARG       # r must be > 0
    assert pool(g.POOL_PP, (float("nan"), 4.0)) == g.ERR_INVALID_ARG
    for kind in (g.POOL_COV, g.POOL_FNS, g.POOL_MEDIAN):
        assert pool(kind, None, ws_bytes=16) == g.ERR_WORKSPACE    # checked before any launch


def test_batch_plan_validation_on_host(g):
    p = g.make_params()
    x = (g.Plane * 2)(_plane(g, 100, 120), _plane(g, 50, 60))
    out = ctypes.c_void_p()
    p97 = g.make_params(flags=g.FLAG_PYRAMID_97)  # the persistent batch kernel fuses the 2x2 pyramid
    assert g.lib.gbssim_batch_plan(x, x, 2, ctypes.byref(p97), 1, None, ctypes.byref(out)) == g.ERR_UNSUPPORTED
    assert g.lib.gbssim_batch_plan(x, x, 0, ctypes.byref(p), 0, None, ctypes.byref(out)) == g.ERR_INVALID_ARG
    p7 = g.make_params(k=7, sigma=1.0)
    assert g.lib.gbssim_batch_plan(x, x, 2, ctypes.byref(p7), 0, None, ctypes.byref(out)) == g.ERR_UNSUPPORTED
    p2 = g.make_params(stride=2)
    assert g.lib.gbssim_batch_plan(x, x, 2, ctypes.byref(p2), 0, None, ctypes.byref(out)) == g.ERR_UNSUPPORTED
    # 50 x 60 halves to 25 x 30, 12 x 15, then 6 x 7 < 11
    assert g.lib.gbssim_batch_plan(x, x, 2, ctypes.byref(p), 1, None, ctypes.byref(out)) == g.ERR_TOO_SMALL
    mixed = (g.Plane * 2)(_plane(g, 100, 120), _plane(g, 50, 60, dtype=3))
    assert g.lib.gbssim_batch_plan(mixed, mixed, 2, ctypes.byref(p), 0, None, ctypes.byref(out)) == g.ERR_INVALID_ARG
    bad = g.Tuning(24, 0, 0, 0)   # rows per item must be a multiple of 16
    assert g.lib.gbssim_batch_plan(x, x, 2, ctypes.byref(p), 0, ctypes.byref(bad), ctypes.byref(out)) \
        == g.ERR_INVALID_ARG
    for tw in (16, 48, 96, 256):  # strips of 32, 64 or 128 columns only
        bad = g.Tuning(0, 0, 0, 0, tw)
        assert g.lib.gbssim_batch_plan(x, x, 2, ctypes.byref(p), 0, ctypes.byref(bad), ctypes.byref(out)) \
            == g.ERR_INVALID_ARG
    assert out.value is None


def test_downscale_factor_matches_oracle(g):
    from oracle import scales

    for h, w in [(1080, 1920), (200, 300), (384, 1000), (383, 1000), (510, 900), (520, 900), (2160, 3840), (1, 1)]:
        assert g.downscale_factor(h, w) == scales.downscale_factor(h, w)
        assert g.downscale_factor(h, w, "ceil_h") == scales.downscale_factor(h, w, "ceil_h")
    assert g.lib.gbssim_downscale_factor(100, 100, 7) == g.ERR_INVALID_ARG
    assert g.lib.gbssim_downscale_factor(0, 100, 0) == g.ERR_INVALID_ARG


def _ws3d(g, x, p, kt, fn="gbssim_msssim3d_workspace_size"):
    n = ctypes.c_size_t()
    rc = getattr(g.lib, fn)(ctypes.byref(x), ctypes.byref(p), int(kt), ctypes.byref(n))
    return rc, n.value


def test_ssim3d_and_msssim3d_validation(g):
    box = dict(window="box")
    v = _plane(g, 1080, 1920, 40)
    rc, n1 = _ws3d(g, v, g.make_params(k=11, **box), 5, "gbssim_ssim3d_workspace_size")
    assert rc == 0 and n1 >= 36 * 16 * 68 * 30 // 2
    rc, n5 = _ws3d(g, v, g.make_params(k=11, **box), 5)
    # the float pyramid of levels 1..4, x and y
    pyr = sum((1080 >> j) * (1920 >> j) for j in range(1, 5)) * 40 * 2 * 4
    assert rc == 0 and n5 >= pyr
    # windows up to 31 x 31 on every level
    assert _ws3d(g, _plane(g, 256, 256, 4), g.make_params(k=32, scales=2, **box), 2)[0] == g.ERR_UNSUPPORTED
    assert _ws3d(g, _plane(g, 256, 256, 4), g.make_params(k=31, scales=1, **box), 2)[0] == 0
    assert _ws3d(g, _plane(g, 256, 256, 4), g.make_params(k=31, scales=2, **box), 2)[0] == 0
    # exact-integer range 5 N^2 (255 4^j)^2 < 2^63 with N = k^2 kt: level 0
    # takes N < 5.3e6 (int64 sums past N = 8256), level 4 N <= 20800
    assert _ws3d(g, _plane(g, 512, 512, 40), g.make_params(k=29, scales=1, **box), 40)[0] == 0
    assert _ws3d(g, _plane(g, 64, 64, 6000), g.make_params(k=31, scales=1, **box), 5600,
                 "gbssim_ssim3d_workspace_size")[0] == g.ERR_UNSUPPORTED
    assert _ws3d(g, _plane(g, 64, 64, 6000), g.make_params(k=31, scales=1, **box), 5500,
                 "gbssim_ssim3d_workspace_size")[0] == 0
    assert _ws3d(g, _plane(g, 512, 512, 40), g.make_params(k=29, scales=5, **box), 24)[0] == 0
    assert _ws3d(g, _plane(g, 512, 512, 40), g.make_params(k=29, scales=5, **box), 25)[0] == g.ERR_UNSUPPORTED
    # levels below k, kt > T, Gaussian windows, other dtypes
    assert _ws3d(g, _plane(g, 100, 100, 4), g.make_params(k=11, scales=5, **box), 2)[0] == g.ERR_TOO_SMALL
    assert _ws3d(g, _plane(g, 100, 100, 4), g.make_params(k=11, scales=3, **box), 5)[0] == g.ERR_TOO_SMALL
    assert _ws3d(g, _plane(g, 100, 100, 4), g.make_params(k=11, scales=2), 2)[0] == g.ERR_UNSUPPORTED
    assert _ws3d(g, _plane(g, 100, 100, 4, dtype=3), g.make_params(k=11, scales=2, **box), 2)[0] == \
        g.ERR_UNSUPPORTED
    assert _ws3d(g, _plane(g, 100, 100, 4), g.make_params(k=11, scales=2, **box), 0)[0] == g.ERR_INVALID_ARG


def test_border_modes_on_host(g):
    x = _plane(g, 7, 9)  # below k = 11: valid windows only are too small, extended ones fit
    for border in ("zero", "reflect"):
        p = g.make_params(border=border)
        rc, n = _ws(g, x, p, g.OP_SSIM)
        assert rc == 0 and n >= 2 * (7 + 10) * (9 + 10)       # the two extended planes
        rc, n = _ws(g, _plane(g, 4, 9), p, g.OP_SSIM)
        assert rc == g.ERR_TOO_SMALL                           # below the mirrored 5 rows
        # five levels of 100 x 100 end at 6 x 6 >= 5
        assert _ws(g, _plane(g, 100, 100), p, g.OP_MSSSIM)[0] == 0
        assert _ws(g, _plane(g, 100, 100), p, g.OP_BACKWARD)[0] == g.ERR_UNSUPPORTED
        xs = (g.Plane * 2)(_plane(g, 100, 120), _plane(g, 50, 60))
        out = ctypes.c_void_p()
        assert g.lib.gbssim_batch_plan(xs, xs, 2, ctypes.byref(p), 0, None, ctypes.byref(out)) == g.ERR_UNSUPPORTED
        pb = g.make_params(window="box", border=border)
        assert _ws3d(g, _plane(g, 64, 64, 4), pb, 2, "gbssim_ssim3d_workspace_size")[0] == g.ERR_UNSUPPORTED
    assert _ws(g, x, g.make_params(), g.OP_SSIM)[0] == g.ERR_TOO_SMALL
    both = g.make_params(flags=g.FLAG_BORDER_ZERO | g.FLAG_BORDER_REFLECT)
    assert _ws(g, x, both, g.OP_SSIM)[0] == g.ERR_INVALID_ARG
    assert g.map_shape(7, 9, g.make_params(border="zero")) == (7, 9)
    assert g.map_shape(1080, 1920, g.make_params(border="reflect", window="box", k=8, stride=4)) == (270, 480)


def _host_ws(g, x, p, chunks):
    n = ctypes.c_size_t(0)
    rc = g.lib.gbssim_msssim_host_workspace_size(ctypes.byref(x), ctypes.byref(p), chunks, ctypes.byref(n))
    return rc, n.value


def test_host_pipeline_plans_on_host(g):
    """gbssim_msssim_host's layouts: chunked mode holds two stages of one
    chunk, streamed mode (chunks = 0) every pair at once plus one arrival
    flag per pair; streamed mode takes only the persistent path's windows."""
    h, w, n = 1080, 1920, 64
    x = _plane(g, h, w, n)
    p = g.make_params()
    pitch_bytes = h * ((w + 15) // 16 * 16)  # uint8 rows padded to 16 bytes
    rc, chunked = _host_ws(g, x, p, 4)
    assert rc == 0 and chunked >= 2 * 2 * 16 * pitch_bytes  # two stages of x and y, 16 pairs each
    rc, streamed = _host_ws(g, x, p, 0)
    assert rc == 0 and streamed >= 2 * n * pitch_bytes + 4 * n + 8 * n
    assert streamed > chunked
    assert _host_ws(g, x, p, -1)[0] == g.ERR_INVALID_ARG
    # chunks above the count are clamped: one chunk per pair
    assert _host_ws(g, _plane(g, h, w, 3), p, 8) == _host_ws(g, _plane(g, h, w, 3), p, 3)
    for kw in (dict(k=7, sigma=1.0), dict(window="box", k=8), dict(stride=2)):
        pk = g.make_params(**kw)
        assert _host_ws(g, x, pk, 4)[0] == 0, kw
        assert _host_ws(g, x, pk, 0)[0] == g.ERR_UNSUPPORTED, kw
    p97 = g.make_params(flags=2)  # GBSSIM_FLAG_PYRAMID_97
    assert _host_ws(g, x, p97, 0)[0] == g.ERR_UNSUPPORTED
    # every level must hold the window, streamed or not
    small = _plane(g, 160, 160, 4)  # level 4 is 10 x 10
    assert _host_ws(g, small, p, 0)[0] == g.ERR_TOO_SMALL
    assert _host_ws(g, small, p, 2)[0] == g.ERR_TOO_SMALL
