"""ctypes binding of libgbssim.so (include/gbssim.h).

Argument marshalling only: every step of SSIM / MS-SSIM runs in the library's
CUDA kernels.  PyTorch supplies device memory (inputs, outputs and the
workspace the C ABI asks for) and the current CUDA stream.  Importing this
module raises ImportError when the library has not been built, so no code path
can silently fall back to a CPU implementation.

Two layers:
  * ``lib`` with the raw C entry points (``lib.gbssim_ssim_map`` ...) and the
    ctypes structs ``Plane`` / ``Params`` mirroring the header;
  * tensor-level helpers with the same names minus the prefix: ``ssim``,
    ``msssim``, ``window_sums``, ``ssim_pool``.  They accept CUDA tensors, or
    CPU tensors (copied to the current CUDA device first, results copied
    back) shaped (H, W), (N, H, W) or (B, C, H, W).
"""
from __future__ import annotations

import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgbssim.so")

if not os.path.exists(LIB_PATH):
    raise ImportError("libgbssim.so is not built; run `python -c 'import __graft_entry__ as g; g.build()'` "
                      "(or paper_2101_06354_gb300/build.py) first")

lib = ctypes.CDLL(LIB_PATH)

MAX_SCALES = 8
MAX_K = 63
MAX_K_BACKWARD = 31
MSSSIM_EXPONENTS = (0.0448, 0.2856, 0.3001, 0.2363, 0.1333)

OK, ERR_INVALID_ARG, ERR_TOO_SMALL, ERR_UNSUPPORTED, ERR_CUDA, ERR_DOMAIN, ERR_TIMEOUT, ERR_WORKSPACE = \
    0, -1, -2, -3, -4, -5, -6, -7
ERR_TOO_LARGE = -8
STATIC_SCRATCH_BYTES = 1 << 20
U8, F16, BF16, F32 = 0, 1, 2, 3
WIN_GAUSSIAN, WIN_BOX = 0, 1
COMBINE_PRODUCT, COMBINE_SUM = 0, 1
OP_SSIM, OP_MSSSIM, OP_BACKWARD, OP_BACKWARD_MS, OP_POOL = 0, 1, 2, 3, 4
POOL_MEAN, POOL_COV, POOL_MINKOWSKI, POOL_DW, POOL_MD, POOL_GM_DSSIM, POOL_HM_DSSIM, POOL_PERCENTILE, \
    POOL_MEDIAN, POOL_FNS, POOL_PP, POOL_GM, POOL_HM, POOL_W_AM, POOL_W_GM, POOL_W_HM, POOL_W_COV = range(17)
POOL_KINDS = {"mean": POOL_MEAN, "cov": POOL_COV, "minkowski": POOL_MINKOWSKI, "dw": POOL_DW, "md": POOL_MD,
              "gm_dssim": POOL_GM_DSSIM, "hm_dssim": POOL_HM_DSSIM, "percentile": POOL_PERCENTILE,
              "median": POOL_MEDIAN, "fns": POOL_FNS, "pp": POOL_PP, "gm": POOL_GM, "hm": POOL_HM,
              "w_am": POOL_W_AM, "w_gm": POOL_W_GM, "w_hm": POOL_W_HM, "w_cov": POOL_W_COV}
FLAG_BOX_TMA = 1


class Tuning(ctypes.Structure):
    _fields_ = [("seg_rows", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32), ("wait_limit", ctypes.c_uint32),
                ("flags", ctypes.c_int32), ("tile_w", ctypes.c_int32)]


TUNING_TEST_STALL = 1
TUNING_TEST_DROP_ARRIVAL = 2


class Plane(ctypes.Structure):
    _fields_ = [("data", ctypes.c_void_p), ("dtype", ctypes.c_int32), ("count", ctypes.c_int32),
                ("height", ctypes.c_int64), ("width", ctypes.c_int64),
                ("row_stride", ctypes.c_int64), ("image_stride", ctypes.c_int64)]


class Params(ctypes.Structure):
    _fields_ = [("window", ctypes.c_int32), ("k", ctypes.c_int32), ("sigma", ctypes.c_double),
                ("K1", ctypes.c_double), ("K2", ctypes.c_double), ("L", ctypes.c_double),
                ("stride", ctypes.c_int32), ("scales", ctypes.c_int32),
                ("exponents", ctypes.c_double * MAX_SCALES), ("combine", ctypes.c_int32),
                ("flags", ctypes.c_int32)]


_P = ctypes.POINTER
_vp, _i32, _i64, _sz = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t
_SIGS = {
    "gbssim_status_string": ([ctypes.c_int], ctypes.c_char_p),
    "gbssim_version": ([], ctypes.c_int),
    "gbssim_params_default": ([_P(Params)], None),
    "gbssim_workspace_size": ([_P(Plane), _P(Params), ctypes.c_int, _P(_sz)], ctypes.c_int),
    "gbssim_ssim_map": ([_P(Plane), _P(Plane), _P(Params), _vp, _i64, _i64, _vp, _vp, _sz, _vp], ctypes.c_int),
    "gbssim_ssim_pool": ([_vp, _i64, _i64, _i64, _i32, _i64, _i32, _vp, _vp, _vp, _sz, _vp], ctypes.c_int),
    "gbssim_msssim": ([_P(Plane), _P(Plane), _P(Params), _vp, _vp, _vp, _sz, _vp], ctypes.c_int),
    "gbssim_window_sums": ([_P(Plane), _P(Plane), _i32, _i32, _vp, _vp], ctypes.c_int),
    "gbssim_window_sums_ex": ([_P(Plane), _P(Plane), _i32, _i32, _i32, _vp, _vp], ctypes.c_int),
    "gbssim_ssim_map_static": ([_P(Plane), _P(Plane), _P(Params), _vp, _i64, _i64, _vp, _vp], ctypes.c_int),
    "gbssim_video_workspace_size": ([_P(Plane), _P(Params), _P(_sz)], ctypes.c_int),
    "gbssim_video": ([_P(Plane), _P(Params), _P(ctypes.c_double), ctypes.c_double, ctypes.c_double, _vp, _vp, _vp,
                      _vp, _sz, _vp], ctypes.c_int),
    "gbssim_batch_plan": ([_P(Plane), _P(Plane), _i32, _P(Params), _i32, _P(Tuning), _P(_vp)], ctypes.c_int),
    "gbssim_batch_workspace_size": ([_vp, _P(_sz)], ctypes.c_int),
    "gbssim_batch_info": ([_vp, _P(_i32), _P(_i32), _P(_i32), _P(_i32)], ctypes.c_int),
    "gbssim_batch_run": ([_vp, _vp, _vp, _vp, _sz, _vp], ctypes.c_int),
    "gbssim_batch_status": ([_vp, _vp, _vp, _vp], ctypes.c_int),
    "gbssim_batch_free": ([_vp], None),
    "gbssim_ssim_backward": ([_P(Plane), _P(Plane), _P(Params), _i32, ctypes.c_double, _vp, _i32, _vp, _vp, _vp,
                              _i32, _i64, _i64, _vp, _vp, _sz, _vp], ctypes.c_int),
    "gbssim_msssim_host_workspace_size": ([_P(Plane), _P(Params), _i32, _P(_sz)], ctypes.c_int),
    "gbssim_series_pool": ([_vp, _i32, _i32, _i64, _i32, _vp, _vp, _vp], ctypes.c_int),
    "gbssim_ssim3d_workspace_size": ([_P(Plane), _P(Params), _i32, _P(_sz)], ctypes.c_int),
    "gbssim_downscale_factor": ([_i64, _i64, _i32], ctypes.c_int),
    "gbssim_downscale": ([_P(Plane), _i32, _vp, _i64, _i64, _vp], ctypes.c_int),
    "gbssim_rgb_to_ycbcr": ([_P(Plane), _P(Plane), _P(Plane), _vp, _vp, _vp, _i64, _i64, _vp], ctypes.c_int),
    "gbssim_loss_saved_size": ([_P(Plane), _P(Params), _i32, _P(_sz)], ctypes.c_int),
    "gbssim_local_mean": ([_P(Plane), _P(Params), _vp, _i64, _i64, _vp], ctypes.c_int),
    "gbssim_ssim_pool_lw": ([_vp, _vp, _i64, _i64, _i64, _i32, _i64, ctypes.c_double, ctypes.c_double, _vp, _vp, _sz,
                             _vp], ctypes.c_int),
    "gbssim_loss_forward": ([_P(Plane), _P(Plane), _P(Params), _i32, _vp, _vp, _vp, _sz, _vp], ctypes.c_int),
    "gbssim_loss_backward": ([_P(Plane), _P(Plane), _P(Params), _i32, ctypes.c_double, _vp, _i32, _vp, _sz, _vp,
                              _i32, _i64, _i64, _vp], ctypes.c_int),
    "gbssim_ssim3d": ([_P(Plane), _P(Plane), _P(Params), _i32, _vp, _vp, _vp, _i64, _i64, _vp, _sz, _vp],
                      ctypes.c_int),
    "gbssim_msssim3d_workspace_size": ([_P(Plane), _P(Params), _i32, _P(_sz)], ctypes.c_int),
    "gbssim_msssim3d": ([_P(Plane), _P(Plane), _P(Params), _i32, _vp, _vp, _vp, _vp, _sz, _vp], ctypes.c_int),
    "gbssim_cmssim_workspace_size": ([_P(Plane), _P(Params), _P(_sz)], ctypes.c_int),
    "gbssim_cmssim": ([_P(Plane), _P(Plane), _P(Params), _vp, _vp, _i64, _i64, _vp, _sz, _vp], ctypes.c_int),
    "gbssim_msssim_host": ([_P(Plane), _P(Plane), _P(Params), _i32, _vp, _vp, _sz, _vp, _vp, _vp], ctypes.c_int),
    "gbssim_fp32_probe": ([_i32, _i32, _i32, _vp, _vp], ctypes.c_int),
    "gbssim_qssim_workspace_size": ([_P(Plane), _P(_sz)], ctypes.c_int),
    "gbssim_qssim": ([_P(Plane), _P(Plane), _P(Params), _vp, _vp, _vp, _sz, _vp], ctypes.c_int),
    "gbssim_msssim_host_ex": ([_P(Plane), _P(Plane), _P(Params), _i32, _P(Tuning), _vp, _vp, _vp, _sz, _vp, _vp,
                               _vp], ctypes.c_int),
}
for _name, (_args, _res) in _SIGS.items():
    _f = getattr(lib, _name)
    _f.argtypes = _args
    _f.restype = _res


class GbssimError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__("%s failed: %s (%d)" % (where, status_string(status), status))


def status_string(status: int) -> str:
    return lib.gbssim_status_string(int(status)).decode()


def _check(rc: int, where: str):
    if rc != OK:
        raise GbssimError(rc, where)


_DTYPES = {torch.uint8: U8, torch.float16: F16, torch.bfloat16: BF16, torch.float32: F32}


FLAG_BORDER_ZERO = 4
FLAG_BORDER_REFLECT = 8
BORDERS = {"valid": 0, "zero": FLAG_BORDER_ZERO, "reflect": FLAG_BORDER_REFLECT}


def make_params(window: str = "gaussian", k: int = 11, sigma: float = 1.5, K1: float = 0.01,
                K2: float = 0.03, L: float = 255.0, stride: int = 1, scales: int = 5,
                exponents=None, combine: str = "product", flags: int = 0, border: str = "valid") -> Params:
    """The C ABI's gbssim_params.  border = "valid" (only windows inside the
    image), "zero" or "reflect" (the image extended by k-1 pixels:
    GBSSIM_FLAG_BORDER_ZERO / _REFLECT)."""
    p = Params()
    lib.gbssim_params_default(ctypes.byref(p))
    p.window = {"gaussian": WIN_GAUSSIAN, "box": WIN_BOX}[window]
    p.k, p.sigma, p.K1, p.K2, p.L, p.stride, p.scales = int(k), float(sigma), float(K1), float(K2), \
        float(L), int(stride), int(scales)
    if exponents is not None:
        if len(exponents) < scales:
            raise ValueError("need one exponent per scale")
        for j in range(MAX_SCALES):
            p.exponents[j] = float(exponents[j]) if j < len(exponents) else 0.0
    p.combine = {"product": COMBINE_PRODUCT, "sum": COMBINE_SUM}[combine]
    p.flags = int(flags) | BORDERS[border]
    return p


def _as_batch(t: torch.Tensor) -> torch.Tensor:
    """View (H, W), (N, H, W) or (B, C, H, W) as (N, H, W) with unit column stride."""
    if t.dim() == 2:
        t = t.unsqueeze(0)
    elif t.dim() == 4:
        t = t.reshape(-1, t.shape[-2], t.shape[-1])
    elif t.dim() != 3:
        raise ValueError("expected a 2-, 3- or 4-D tensor")
    if t.stride(-1) != 1 or (t.shape[0] > 1 and t.stride(0) < t.shape[1] * t.stride(1)):
        t = t.contiguous()
    return t


def plane(t: torch.Tensor) -> Plane:
    """Describe an (N, H, W) CUDA tensor (unit column stride) for the C ABI."""
    if t.dtype not in _DTYPES:
        raise TypeError("unsupported dtype %s" % t.dtype)
    n, h, w = t.shape
    return Plane(t.data_ptr(), _DTYPES[t.dtype], n, h, w, t.stride(1), t.stride(0) if n > 1 else h * t.stride(1))


def _stream(dev) -> int:
    return torch.cuda.current_stream(dev).cuda_stream


def _prepare(x, y):
    host = x.device.type == "cpu"
    dev = torch.device("cuda", torch.cuda.current_device()) if host else x.device
    if host:
        x = x.to(dev, non_blocking=True)
        y = y.to(dev, non_blocking=True)
    if y.device != x.device or y.dtype != x.dtype or y.shape != x.shape:
        raise ValueError("x and y must share device, dtype and shape")
    xb, yb = _as_batch(x), _as_batch(y)
    if xb.stride() != yb.stride():
        xb, yb = xb.contiguous(), yb.contiguous()
    return host, dev, xb, yb


def workspace(px: Plane, p: Params, op: int, dev) -> torch.Tensor:
    n = ctypes.c_size_t()
    _check(lib.gbssim_workspace_size(ctypes.byref(px), ctypes.byref(p), op, ctypes.byref(n)),
           "gbssim_workspace_size")
    return torch.empty(max(int(n.value), 1), dtype=torch.uint8, device=dev)


def map_shape(h: int, w: int, p: Params):
    """(OH, OW) of the SSIM map for params p (border modes extend by k-1)."""
    ext = p.k - 1 if p.flags & (FLAG_BORDER_ZERO | FLAG_BORDER_REFLECT) else 0
    return out_shape(h + ext, w + ext, p.k, p.stride)


def out_shape(h: int, w: int, k: int, stride: int):
    return ((h - k) // stride + 1, (w - k) // stride + 1)


def ssim(x: torch.Tensor, y: torch.Tensor, return_map: bool = False, ws: torch.Tensor = None, **kw):
    """MSSIM of each pair (float64 tensor of length N), optionally with the
    float Q map (N, OH, OW).  Keyword arguments as ``make_params``."""
    host, dev, xb, yb = _prepare(x, y)
    p = make_params(**kw)
    px, py = plane(xb), plane(yb)
    n = xb.shape[0]
    if ws is None:
        ws = workspace(px, p, OP_SSIM, dev)
    mean = torch.empty(n, dtype=torch.float64, device=dev)
    mp = None
    if return_map:
        oh, ow = map_shape(xb.shape[1], xb.shape[2], p)
        mp = torch.empty((n, oh, ow), dtype=torch.float32, device=dev)
    _check(lib.gbssim_ssim_map(ctypes.byref(px), ctypes.byref(py), ctypes.byref(p),
                               mp.data_ptr() if mp is not None else None,
                               mp.stride(1) if mp is not None else 0,
                               mp.stride(0) if mp is not None else 0,
                               mean.data_ptr(), ws.data_ptr(), ws.numel(), _stream(dev)),
           "gbssim_ssim_map")
    if host:
        mean = mean.cpu()
        mp = mp.cpu() if mp is not None else None
    return (mean, mp) if return_map else mean


def ssim_static(x: torch.Tensor, y: torch.Tensor, return_map: bool = False, **kw):
    """As ``ssim`` but through gbssim_ssim_map_static, which needs no
    workspace: its scratch is a static device array inside the library, for
    callers that cannot allocate device memory.  Calls whose GPU work overlaps
    race on that array."""
    host, dev, xb, yb = _prepare(x, y)
    p = make_params(**kw)
    px, py = plane(xb), plane(yb)
    n = xb.shape[0]
    mean = torch.empty(n, dtype=torch.float64, device=dev)
    mp = None
    if return_map:
        oh, ow = map_shape(xb.shape[1], xb.shape[2], p)
        mp = torch.empty((n, oh, ow), dtype=torch.float32, device=dev)
    _check(lib.gbssim_ssim_map_static(ctypes.byref(px), ctypes.byref(py), ctypes.byref(p),
                                      mp.data_ptr() if mp is not None else None,
                                      mp.stride(1) if mp is not None else 0,
                                      mp.stride(0) if mp is not None else 0,
                                      mean.data_ptr(), _stream(dev)),
           "gbssim_ssim_map_static")
    if host:
        mean = mean.cpu()
        mp = mp.cpu() if mp is not None else None
    return (mean, mp) if return_map else mean


_side_streams = {}


def _copy_stream(dev, which: int = 0) -> torch.cuda.Stream:
    """Side streams of the host pipeline (0: copies, 1: second compute stream)."""
    key = (dev, which)
    if key not in _side_streams:
        _side_streams[key] = torch.cuda.Stream(device=dev)
    return _side_streams[key]


def host_workspace(x: torch.Tensor, chunks: int, **kw) -> torch.Tensor:
    """Device workspace for msssim_host on host planes shaped like x."""
    kw.setdefault("exponents", MSSSIM_EXPONENTS[: kw.get("scales", 5)])
    p = make_params(**kw)
    px = plane(_as_batch(x))
    nb = ctypes.c_size_t()
    _check(lib.gbssim_msssim_host_workspace_size(ctypes.byref(px), ctypes.byref(p), int(chunks), ctypes.byref(nb)),
           "gbssim_msssim_host_workspace_size")
    return torch.empty(max(int(nb.value), 1), dtype=torch.uint8, device=torch.device("cuda", torch.cuda.current_device()))


def msssim_host(x: torch.Tensor, y: torch.Tensor, chunks: int = 4, ws: torch.Tensor = None,
                out: torch.Tensor = None, sync: bool = True, two_compute_streams: bool = False,
                tuning: "Tuning" = None, status: torch.Tensor = None, **kw) -> torch.Tensor:
    """MS-SSIM of pairs held in host memory (gbssim_msssim_host): chunks of
    the batch are copied on a side stream while the previous chunk is scored
    on the current stream; chunks=0 streams instead (one launch over all
    pairs, each group of pairs scored as soon as its copy lands; equal to the
    device call up to fp32 summation order).  Returns a pinned CPU
    float64 tensor of length N, valid at return when sync=True (else once the
    current stream completes).  x and y should be pinned for the copies to
    overlap.  ``tuning`` (a Tuning: wait_limit, test flags) and ``status``
    (a pinned int32 CPU tensor of one element that receives the launch's
    status word) go through gbssim_msssim_host_ex; streamed mode only."""
    if x.device.type != "cpu" or y.device.type != "cpu":
        raise ValueError("msssim_host takes host tensors")
    if y.dtype != x.dtype or y.shape != x.shape:
        raise ValueError("x and y must share dtype and shape")
    dev = torch.device("cuda", torch.cuda.current_device())
    xb, yb = _as_batch(x), _as_batch(y)
    if xb.stride() != yb.stride():
        xb, yb = xb.contiguous(), yb.contiguous()
    kw.setdefault("exponents", MSSSIM_EXPONENTS[: kw.get("scales", 5)])
    p = make_params(**kw)
    px, py = plane(xb), plane(yb)
    n = xb.shape[0]
    if ws is None:
        ws = host_workspace(xb, chunks, **kw)
    if out is None:
        out = torch.empty(n, dtype=torch.float64, pin_memory=True)
    cs, s2 = _copy_stream(dev, 0), _copy_stream(dev, 1)
    if tuning is not None or status is not None:
        if status is not None and (status.device.type != "cpu" or status.dtype != torch.int32 or status.numel() < 1):
            raise ValueError("status must be a CPU int32 tensor")
        _check(lib.gbssim_msssim_host_ex(ctypes.byref(px), ctypes.byref(py), ctypes.byref(p), int(chunks),
                                         ctypes.byref(tuning) if tuning is not None else None, out.data_ptr(),
                                         status.data_ptr() if status is not None else None, ws.data_ptr(),
                                         ws.numel(), _stream(dev), cs.cuda_stream,
                                         s2.cuda_stream if two_compute_streams else None), "gbssim_msssim_host_ex")
    else:
        _check(lib.gbssim_msssim_host(ctypes.byref(px), ctypes.byref(py), ctypes.byref(p), int(chunks),
                                      out.data_ptr(), ws.data_ptr(), ws.numel(), _stream(dev), cs.cuda_stream,
                                      s2.cuda_stream if two_compute_streams else None), "gbssim_msssim_host")
    if sync:
        torch.cuda.current_stream(dev).synchronize()
    return out


def msssim(x: torch.Tensor, y: torch.Tensor, per_scale: bool = False, ws: torch.Tensor = None, **kw):
    """MS-SSIM of each pair (float64 tensor of length N); with per_scale=True
    also the (N, scales, 2) tensor of (mean cs_j, mean Q_j).  Host tensors go
    through msssim_host (copies overlapped with compute) unless per_scale is
    asked for."""
    if x.device.type == "cpu" and y.device.type == "cpu" and not per_scale:
        return msssim_host(x, y, **kw)
    host, dev, xb, yb = _prepare(x, y)
    kw.setdefault("exponents", MSSSIM_EXPONENTS[: kw.get("scales", 5)])
    if kw.pop("pyramid", "avg2") == "97":
        kw["flags"] = kw.get("flags", 0) | FLAG_PYRAMID_97
    p = make_params(**kw)
    px, py = plane(xb), plane(yb)
    n = xb.shape[0]
    if ws is None:
        ws = workspace(px, p, OP_MSSSIM, dev)
    score = torch.empty(n, dtype=torch.float64, device=dev)
    per = torch.empty((n, p.scales, 2), dtype=torch.float64, device=dev) if per_scale else None
    _check(lib.gbssim_msssim(ctypes.byref(px), ctypes.byref(py), ctypes.byref(p), score.data_ptr(),
                             per.data_ptr() if per is not None else None, ws.data_ptr(), ws.numel(),
                             _stream(dev)), "gbssim_msssim")
    if host:
        score = score.cpu()
        per = per.cpu() if per is not None else None
    return (score, per) if per_scale else score


def window_sums(x: torch.Tensor, y: torch.Tensor, k: int, stride: int = 1, flags: int = 0) -> torch.Tensor:
    """Exact int64 window sums (N, OH, OW, 5) of a uint8 pair batch."""
    host, dev, xb, yb = _prepare(x, y)
    n, h, w = xb.shape
    oh, ow = out_shape(h, w, k, stride)
    out = torch.empty((n, max(oh, 0), max(ow, 0), 5), dtype=torch.int64, device=dev)
    px, py = plane(xb), plane(yb)
    _check(lib.gbssim_window_sums_ex(ctypes.byref(px), ctypes.byref(py), int(k), int(stride), int(flags),
                                     out.data_ptr(), _stream(dev)), "gbssim_window_sums_ex")
    return out.cpu() if host else out


def ssim_pool(qmap: torch.Tensor, kind: str = "mean", *args: float, ws: torch.Tensor = None) -> torch.Tensor:
    """Pool float maps (H, W) or (N, H, W) into one double each.  kind is a
    key of POOL_KINDS; args are its parameters: minkowski / dw (p),
    md (p, o), percentile (p), pp (p, r)."""
    m = qmap if qmap.dim() == 3 else qmap.unsqueeze(0)
    if m.dtype != torch.float32 or m.stride(-1) != 1:
        raise TypeError("expected float32 maps with unit column stride")
    n, h, w = m.shape
    dev = m.device
    px = Plane(m.data_ptr(), F32, n, h, w, m.stride(1), m.stride(0) if n > 1 else h * m.stride(1))
    if ws is None:
        ws = workspace(px, Params(), OP_POOL, dev)
    out = torch.empty(n, dtype=torch.float64, device=dev)
    a = (ctypes.c_double * 2)(*(list(map(float, args)) + [0.0, 0.0])[:2]) if args else None
    _check(lib.gbssim_ssim_pool(m.data_ptr(), h, w, m.stride(1), n, px.image_stride, POOL_KINDS[kind], a,
                                out.data_ptr(), ws.data_ptr(), ws.numel(), _stream(dev)), "gbssim_ssim_pool")
    return out


def local_mean(x: torch.Tensor, **kw) -> torch.Tensor:
    """Window-weighted local mean (gbssim_local_mean) of (H, W) or (N, H, W)
    CUDA planes at every valid strided position; keyword arguments as
    make_params (window, k, sigma, stride)."""
    xb = _as_batch(x)
    p = make_params(**kw)
    n, h, w = xb.shape
    oh, ow = out_shape(h, w, p.k, p.stride)
    out = torch.empty((n, oh, ow), dtype=torch.float32, device=xb.device)
    px = plane(xb)
    _check(lib.gbssim_local_mean(ctypes.byref(px), ctypes.byref(p), out.data_ptr(), ow, oh * ow, _stream(xb.device)),
           "gbssim_local_mean")
    return out if x.dim() != 2 else out[0]


def ssim_pool_lw(qmap: torch.Tensor, mu_ref: torch.Tensor, a: float, b: float) -> torch.Tensor:
    """Luminance-weighted pooling (gbssim_ssim_pool_lw) of float maps with the
    reference's local-mean maps of the same shape."""
    m = qmap if qmap.dim() == 3 else qmap.unsqueeze(0)
    u = mu_ref if mu_ref.dim() == 3 else mu_ref.unsqueeze(0)
    m, u = m.contiguous(), u.contiguous()
    if m.shape != u.shape or m.dtype != torch.float32 or u.dtype != torch.float32:
        raise ValueError("expected float32 maps of one shape")
    n, h, w = m.shape
    px = Plane(m.data_ptr(), F32, n, h, w, w, h * w)
    ws = workspace(px, Params(), OP_POOL, m.device)
    out = torch.empty(n, dtype=torch.float64, device=m.device)
    _check(lib.gbssim_ssim_pool_lw(m.data_ptr(), u.data_ptr(), h, w, w, n, h * w, float(a), float(b), out.data_ptr(),
                                   ws.data_ptr(), ws.numel(), _stream(m.device)), "gbssim_ssim_pool_lw")
    return out


def series_pool(scores: torch.Tensor, kind: str = "mean", *args: float) -> torch.Tensor:
    """Temporal pooling (gbssim_series_pool) of frame-score series (T,) or
    (N, T) on the GPU into one double each.  kind is a key of POOL_KINDS;
    args as for ssim_pool, and k for the windowed kinds w_am, w_gm, w_hm,
    w_cov."""
    s = scores if scores.dim() == 2 else scores.unsqueeze(0)
    if s.dtype != torch.float64 or s.device.type != "cuda" or s.stride(-1) != 1:
        raise TypeError("expected float64 CUDA series with unit stride")
    n_series, t = s.shape
    out = torch.empty(n_series, dtype=torch.float64, device=s.device)
    a = (ctypes.c_double * 2)(*(list(map(float, args)) + [0.0, 0.0])[:2]) if args else None
    _check(lib.gbssim_series_pool(s.data_ptr(), t, n_series, s.stride(0) if n_series > 1 else t, POOL_KINDS[kind], a,
                                  out.data_ptr(), _stream(s.device)), "gbssim_series_pool")
    return out


def ssim3d(x: torch.Tensor, y: torch.Tensor, kt: int = 5, k: int = 11, return_map: bool = False,
           ws: torch.Tensor = None, **kw):
    """SSIM-3D (gbssim_ssim3d) of a uint8 video pair (T, H, W): k x k x kt
    rectangular windows.  Returns (video score, per-frame scores of the T-kt+1
    output frames[, maps])."""
    if x.dtype != torch.uint8 or x.dim() != 3 or y.shape != x.shape or y.dtype != x.dtype:
        raise ValueError("expected two uint8 videos (T, H, W) of one shape")
    dev = x.device
    xb, yb = x.contiguous(), y.contiguous()
    p = make_params(window="box", k=k, **kw)
    px, py = plane(xb), plane(yb)
    T, H, W = x.shape
    if ws is None:
        nb = ctypes.c_size_t()
        _check(lib.gbssim_ssim3d_workspace_size(ctypes.byref(px), ctypes.byref(p), int(kt), ctypes.byref(nb)),
               "gbssim_ssim3d_workspace_size")
        ws = torch.empty(max(int(nb.value), 1), dtype=torch.uint8, device=dev)
    frames = torch.empty(T - kt + 1, dtype=torch.float64, device=dev)
    score = torch.empty(1, dtype=torch.float64, device=dev)
    qmap = torch.empty((T - kt + 1, H - k + 1, W - k + 1), dtype=torch.float32, device=dev) if return_map else None
    _check(lib.gbssim_ssim3d(ctypes.byref(px), ctypes.byref(py), ctypes.byref(p), int(kt), frames.data_ptr(),
                             score.data_ptr(), qmap.data_ptr() if return_map else None, W - k + 1,
                             (H - k + 1) * (W - k + 1), ws.data_ptr(), ws.numel(), _stream(dev)), "gbssim_ssim3d")
    return (score[0], frames, qmap) if return_map else (score[0], frames)


def msssim3d(x: torch.Tensor, y: torch.Tensor, kt: int = 5, k: int = 11, per_scale: bool = False,
             ws: torch.Tensor = None, **kw):
    """MS-SSIM-3D (gbssim_msssim3d) of a uint8 video pair (T, H, W): SSIM-3D
    with k x k x kt windows on every level of the frames' 2x2 pyramid,
    combined per output frame like MS-SSIM.  Returns (video score, per-frame
    scores[, (T-kt+1, scales, 2) of (mean cs_j, mean Q_j)])."""
    if x.dtype != torch.uint8 or x.dim() != 3 or y.shape != x.shape or y.dtype != x.dtype:
        raise ValueError("expected two uint8 videos (T, H, W) of one shape")
    dev = x.device
    xb, yb = x.contiguous(), y.contiguous()
    kw.setdefault("exponents", MSSSIM_EXPONENTS[: kw.get("scales", 5)])
    p = make_params(window="box", k=k, **kw)
    px, py = plane(xb), plane(yb)
    T = x.shape[0]
    if ws is None:
        nb = ctypes.c_size_t()
        _check(lib.gbssim_msssim3d_workspace_size(ctypes.byref(px), ctypes.byref(p), int(kt), ctypes.byref(nb)),
               "gbssim_msssim3d_workspace_size")
        ws = torch.empty(max(int(nb.value), 1), dtype=torch.uint8, device=dev)
    frames = torch.empty(T - kt + 1, dtype=torch.float64, device=dev)
    score = torch.empty(1, dtype=torch.float64, device=dev)
    per = torch.empty((T - kt + 1, p.scales, 2), dtype=torch.float64, device=dev) if per_scale else None
    _check(lib.gbssim_msssim3d(ctypes.byref(px), ctypes.byref(py), ctypes.byref(p), int(kt), frames.data_ptr(),
                               score.data_ptr(), per.data_ptr() if per_scale else None, ws.data_ptr(), ws.numel(),
                               _stream(dev)), "gbssim_msssim3d")
    return (score[0], frames, per) if per_scale else (score[0], frames)


FLAG_PYRAMID_97 = 2
DOWNSCALE_RULES = {"round_min": 0, "ceil_h": 1}


def downscale_factor(h: int, w: int, rule: str = "round_min") -> int:
    """Automatic downscaling factor Z (gbssim_downscale_factor)."""
    z = lib.gbssim_downscale_factor(int(h), int(w), DOWNSCALE_RULES[rule])
    _check(OK if z > 0 else z, "gbssim_downscale_factor")
    return z


def downscale(x: torch.Tensor, z: int) -> torch.Tensor:
    """Z x Z block means (gbssim_downscale) of (H, W) or (N, H, W) planes on
    the GPU into float32 (N, H // z, W // z)."""
    xb = _as_batch(x)
    if xb.device.type != "cuda":
        raise ValueError("downscale takes CUDA tensors")
    n, h, w = xb.shape
    out = torch.empty((n, h // z, w // z), dtype=torch.float32, device=xb.device)
    px = plane(xb)
    _check(lib.gbssim_downscale(ctypes.byref(px), int(z), out.data_ptr(), w // z, (h // z) * (w // z),
                                _stream(xb.device)), "gbssim_downscale")
    return out if x.dim() != 2 else out[0]


def rgb_to_ycbcr(r: torch.Tensor, g: torch.Tensor, b: torch.Tensor):
    """BT.709 Y, Cb, Cr float planes (gbssim_rgb_to_ycbcr) of planar RGB
    CUDA tensors (H, W) or (N, H, W)."""
    rb, gb, bb = _as_batch(r).contiguous(), _as_batch(g).contiguous(), _as_batch(b).contiguous()
    n, h, w = rb.shape
    out = torch.empty((3, n, h, w), dtype=torch.float32, device=rb.device)
    pr, pg, pb = plane(rb), plane(gb), plane(bb)
    _check(lib.gbssim_rgb_to_ycbcr(ctypes.byref(pr), ctypes.byref(pg), ctypes.byref(pb), out[0].data_ptr(),
                                   out[1].data_ptr(), out[2].data_ptr(), w, h * w, _stream(rb.device)),
           "gbssim_rgb_to_ycbcr")
    return out[0], out[1], out[2]


def colour_ssim(ref_rgb, dis_rgb, weights=(0.8, 0.1, 0.1), **kw):
    """Channel-weighted colour SSIM of planar RGB frames (Section
    "Channel-wise SSIM"): BT.709 Y, Cb, Cr of both, SSIM of each plane, frame
    score (w_Y S_Y + w_Cb S_Cb + w_Cr S_Cr) / (w_Y + w_Cb + w_Cr).  ref_rgb and
    dis_rgb are (R, G, B) tuples of CUDA tensors (frames, H, W).  Returns
    gbssim_video's (frame_scores, plane_scores, (mean, p10, pp)).  The paper's
    tuned weights are 1, -0.3, -0.3."""
    xs = rgb_to_ycbcr(*ref_rgb)
    ys = rgb_to_ycbcr(*dis_rgb)
    return video_ssim(xs, ys, weights=weights, **kw)


def enhanced_ssim(x: torch.Tensor, y: torch.Tensor, z: int = None, rule: str = "round_min", k: int = 11,
                  stride: int = 5, return_map: bool = False, **kw):
    """Enhanced SSIM (the paper's recommended variant, Concluding section):
    luminance planes, z x z block-mean downscaling (gbssim_downscale; z
    from gbssim_downscale_factor's `rule` when not given), k x k rectangular
    windows at the given stride (exact integer window sums on uint8 input
    when z = 1), and coefficient-of-variation pooling of each Q map
    (gbssim_ssim_pool).  (H, W) or (N, H, W) CUDA tensors; returns the CoV
    score per pair (float64, N)[, and the Q maps]."""
    xb, yb = _as_batch(x), _as_batch(y)
    if z is None:
        z = downscale_factor(xb.shape[1], xb.shape[2], rule)
    if z > 1:
        xb, yb = downscale(xb, z), downscale(yb, z)
    _, q = ssim(xb, yb, return_map=True, window="box", k=k, stride=stride, **kw)
    score = ssim_pool(q, "cov")
    return (score, q) if return_map else score


def cmssim(ref_rgb, dis_rgb, return_map: bool = False, ws: torch.Tensor = None, **kw):
    """CMSSIM (gbssim_cmssim) of RGB pairs: ref_rgb and dis_rgb are (R, G, B)
    tuples of CUDA tensors (H, W) or (N, H, W), linear RGB in [0, 1] (uint8
    values are divided by 255).  Keyword arguments as make_params (Gaussian
    window k, sigma; K1, K2; stride).  Returns the score per pair (float64,
    N)[, and the weighted maps]."""
    xs = [_as_batch(t).contiguous() for t in ref_rgb]
    ys = [_as_batch(t).contiguous() for t in dis_rgb]
    if len(xs) != 3 or len(ys) != 3:
        raise ValueError("expected (R, G, B) planes")
    dev = xs[0].device
    p = make_params(**kw)
    px = (Plane * 3)(*[plane(t) for t in xs])
    py = (Plane * 3)(*[plane(t) for t in ys])
    n, h, w = xs[0].shape
    if ws is None:
        nb = ctypes.c_size_t()
        _check(lib.gbssim_cmssim_workspace_size(ctypes.byref(px[0]), ctypes.byref(p), ctypes.byref(nb)),
               "gbssim_cmssim_workspace_size")
        ws = torch.empty(max(int(nb.value), 1), dtype=torch.uint8, device=dev)
    score = torch.empty(n, dtype=torch.float64, device=dev)
    mp = None
    if return_map:
        oh, ow = out_shape(h, w, p.k, p.stride)
        mp = torch.empty((n, oh, ow), dtype=torch.float32, device=dev)
    _check(lib.gbssim_cmssim(px, py, ctypes.byref(p), score.data_ptr(), mp.data_ptr() if mp is not None else None,
                             mp.stride(1) if mp is not None else 0, mp.stride(0) if mp is not None else 0,
                             ws.data_ptr(), ws.numel(), _stream(dev)), "gbssim_cmssim")
    return (score, mp) if return_map else score


def qssim(ref, dis, return_terms: bool = False, ws: torch.Tensor = None, **kw):
    """QSSIM (gbssim_qssim) of colour pairs: ref and dis are 3-tuples of CUDA
    tensors (H, W) or (N, H, W), the tristimulus planes (RGB, YUV, ...) of
    one dtype and shape.  Keyword arguments K1, K2, L as make_params.
    Returns the score per pair (float64, N)[, and (N, 2) luminance and
    contrast-structure factors]."""
    xs = [_as_batch(t).contiguous() for t in ref]
    ys = [_as_batch(t).contiguous() for t in dis]
    if len(xs) != 3 or len(ys) != 3:
        raise ValueError("expected three planes per picture")
    dev = xs[0].device
    p = make_params(**kw)
    px = (Plane * 3)(*[plane(t) for t in xs])
    py = (Plane * 3)(*[plane(t) for t in ys])
    n = xs[0].shape[0]
    if ws is None:
        nb = ctypes.c_size_t()
        _check(lib.gbssim_qssim_workspace_size(ctypes.byref(px[0]), ctypes.byref(nb)), "gbssim_qssim_workspace_size")
        ws = torch.empty(max(int(nb.value), 1), dtype=torch.uint8, device=dev)
    score = torch.empty(n, dtype=torch.float64, device=dev)
    terms = torch.empty((n, 2), dtype=torch.float64, device=dev) if return_terms else None
    _check(lib.gbssim_qssim(px, py, ctypes.byref(p), score.data_ptr(),
                            terms.data_ptr() if terms is not None else None, ws.data_ptr(), ws.numel(),
                            _stream(dev)), "gbssim_qssim")
    return (score, terms) if return_terms else score


_GDT = {torch.float32: F32, torch.float16: F16, torch.bfloat16: BF16}


def ssim_backward(x: torch.Tensor, y: torch.Tensor, multiscale: bool = False, grad_scale: float = 1.0,
                  grad_out: torch.Tensor = None, grad_dtype=None, return_score: bool = False,
                  ws: torch.Tensor = None, fwd_score: torch.Tensor = None, fwd_per_scale: torch.Tensor = None,
                  **kw):
    """d score / d y for each pair (gbssim_ssim_backward), shaped like y.

    score is MSSIM (multiscale=False) or MS-SSIM.  The result is multiplied by
    ``grad_scale`` and, when given, by the device float64 tensor ``grad_out``
    (one element, or one per pair).  ``grad_dtype`` defaults to y's dtype for
    floating inputs and float32 for uint8."""
    host, dev, xb, yb = _prepare(x, y)
    if multiscale:
        kw.setdefault("exponents", MSSSIM_EXPONENTS[: kw.get("scales", 5)])
    p = make_params(**kw)
    px, py = plane(xb), plane(yb)
    n, h, w = xb.shape
    gdt = grad_dtype or (y.dtype if y.dtype in _GDT else torch.float32)
    grad = torch.empty((n, h, w), dtype=gdt, device=dev)
    if ws is None:
        ws = workspace(px, p, OP_BACKWARD_MS if multiscale else OP_BACKWARD, dev)
    score = torch.empty(n, dtype=torch.float64, device=dev) if return_score else None
    go = None
    if grad_out is not None:
        go = grad_out.detach().to(device=dev, dtype=torch.float64).contiguous().reshape(-1)
        if go.numel() not in (1, n):
            raise ValueError("grad_out must have 1 or N elements")
    if (fwd_score is None) != (fwd_per_scale is None):
        raise ValueError("fwd_score and fwd_per_scale go together")
    fs = fwd_score.contiguous() if fwd_score is not None else None
    fp = fwd_per_scale.contiguous() if fwd_per_scale is not None else None
    _check(lib.gbssim_ssim_backward(ctypes.byref(px), ctypes.byref(py), ctypes.byref(p), int(bool(multiscale)),
                                    float(grad_scale), go.data_ptr() if go is not None else None,
                                    int(go is not None and go.numel() == n and n > 1),
                                    fs.data_ptr() if fs is not None else None,
                                    fp.data_ptr() if fp is not None else None, grad.data_ptr(),
                                    _GDT[gdt], grad.stride(1), grad.stride(0),
                                    score.data_ptr() if score is not None else None,
                                    ws.data_ptr(), ws.numel(), _stream(dev)), "gbssim_ssim_backward")
    grad = grad.reshape(y.shape)
    if host:
        grad = grad.cpu()
        score = score.cpu() if score is not None else None
    return (grad, score) if return_score else grad


class _SSIMLossFn(torch.autograd.Function):
    """loss = 1 - mean over pairs of SSIM (or MS-SSIM); gradient w.r.t. y only
    (x is the reference).

    recompute=True (the default): the forward is the plain score call
    (gbssim_ssim_map, or gbssim_msssim with its per-scale means) and keeps
    only x, y and the pooled values; the backward (gbssim_ssim_backward)
    recomputes every level's window moments, forms the coefficient maps in a
    transient workspace and runs the gradient kernels.
    recompute=False: the forward (gbssim_loss_forward) runs each level once in
    coefficient mode and keeps the coefficient maps, the pyramid and the
    pooled values in a device buffer (12 bytes per output position per
    level); the backward (gbssim_loss_backward) runs only the gradient
    kernels from it."""

    @staticmethod
    def forward(ctx, x, y, multiscale, recompute, kw):
        xb, yb = _as_batch(x), _as_batch(y)
        if xb.stride() != yb.stride():
            xb, yb = xb.contiguous(), yb.contiguous()
        kw = dict(kw)
        if multiscale:
            kw.setdefault("exponents", MSSSIM_EXPONENTS[: kw.get("scales", 5)])
        p = make_params(**kw)
        px, py = plane(xb), plane(yb)
        dev = xb.device
        n = xb.shape[0]
        score = torch.empty(n, dtype=torch.float64, device=dev)
        if recompute:
            per = None
            if multiscale:
                per = torch.empty((n, p.scales, 2), dtype=torch.float64, device=dev)
                ws = workspace(px, p, OP_MSSSIM, dev)
                _check(lib.gbssim_msssim(ctypes.byref(px), ctypes.byref(py), ctypes.byref(p), score.data_ptr(),
                                         per.data_ptr(), ws.data_ptr(), ws.numel(), _stream(dev)), "gbssim_msssim")
                ctx.save_for_backward(xb, yb, score, per)
            else:
                ws = workspace(px, p, OP_SSIM, dev)
                _check(lib.gbssim_ssim_map(ctypes.byref(px), ctypes.byref(py), ctypes.byref(p), None, 0, 0,
                                           score.data_ptr(), ws.data_ptr(), ws.numel(), _stream(dev)),
                       "gbssim_ssim_map")
                ctx.save_for_backward(xb, yb)
        else:
            nb = ctypes.c_size_t()
            _check(lib.gbssim_loss_saved_size(ctypes.byref(px), ctypes.byref(p), int(multiscale),
                                              ctypes.byref(nb)), "gbssim_loss_saved_size")
            saved = torch.empty(max(int(nb.value), 1), dtype=torch.uint8, device=dev)
            _check(lib.gbssim_loss_forward(ctypes.byref(px), ctypes.byref(py), ctypes.byref(p), int(multiscale),
                                           score.data_ptr(), None, saved.data_ptr(), saved.numel(), _stream(dev)),
                   "gbssim_loss_forward")
            ctx.save_for_backward(xb, yb, saved)
        ctx.multiscale = multiscale
        ctx.recompute = recompute
        ctx.params = p
        ctx.y_shape = y.shape
        ctx.n = n
        return 1.0 - score.mean()

    @staticmethod
    def backward(ctx, grad_loss):
        if not ctx.needs_input_grad[1]:
            return None, None, None, None, None
        xb, yb = ctx.saved_tensors[:2]
        n, h, w = yb.shape
        dev = yb.device
        g = torch.empty((n, h, w), dtype=yb.dtype, device=dev)
        go = grad_loss.to(torch.float64).contiguous()
        px, py = plane(xb), plane(yb)
        p = ctx.params
        if ctx.recompute:
            fs = fp = None
            if ctx.multiscale:
                fs, fp = ctx.saved_tensors[2], ctx.saved_tensors[3]
            ws = workspace(px, p, OP_BACKWARD_MS if ctx.multiscale else OP_BACKWARD, dev)
            _check(lib.gbssim_ssim_backward(ctypes.byref(px), ctypes.byref(py), ctypes.byref(p),
                                            int(ctx.multiscale), -1.0 / ctx.n, go.data_ptr(), 0,
                                            fs.data_ptr() if fs is not None else None,
                                            fp.data_ptr() if fp is not None else None, g.data_ptr(),
                                            _GDT[yb.dtype], w, h * w, None, ws.data_ptr(), ws.numel(),
                                            _stream(dev)), "gbssim_ssim_backward")
        else:
            saved = ctx.saved_tensors[2]
            _check(lib.gbssim_loss_backward(ctypes.byref(px), ctypes.byref(py), ctypes.byref(p),
                                            int(ctx.multiscale), -1.0 / ctx.n, go.data_ptr(), 0, saved.data_ptr(),
                                            saved.numel(), g.data_ptr(), _GDT[yb.dtype], w, h * w, _stream(dev)),
                   "gbssim_loss_backward")
        return None, g.reshape(ctx.y_shape), None, None, None


class SSIMLoss(torch.nn.Module):
    """1 - SSIM (or MS-SSIM with multiscale=True) averaged over the batch,
    differentiable with respect to the second argument.  Inputs (H, W),
    (N, H, W) or (B, C, H, W) float tensors on a CUDA device; keyword
    arguments as ``make_params`` (e.g. L=1.0 for inputs in [0, 1]).

    recompute=True (default): the backward recomputes the window moments from
    x and y (nothing but the pooled scores is kept between forward and
    backward); recompute=False keeps every level's coefficient maps from the
    forward instead (faster backward, 12 bytes per output position per level
    held until the backward)."""

    def __init__(self, multiscale: bool = False, recompute: bool = True, **kw):
        super().__init__()
        self.multiscale = multiscale
        self.recompute = recompute
        self.kw = kw

    def forward(self, x: torch.Tensor, y: torch.Tensor) -> torch.Tensor:
        return _SSIMLossFn.apply(x.detach(), y, self.multiscale, self.recompute, dict(self.kw))


def video_ssim(xs, ys, weights=(6.0, 1.0, 1.0), percentile: float = 10.0, pp_r: float = 4.0, **kw):
    """Colour + temporal SSIM of a YUV video (gbssim_video).  xs = (Y, U, V)
    reference planes and ys = (Y, U, V) distorted planes, each a CUDA tensor
    (frames, H_p, W_p).  Returns (frame_scores, plane_scores (3, frames),
    (mean, percentile, percentile_pooled))."""
    if len(xs) != 3 or len(ys) != 3:
        raise ValueError("expected (Y, U, V) planes")
    pl = []
    keep = []
    for a, b in zip(xs, ys):
        a, b = _as_batch(a), _as_batch(b)
        if a.stride() != b.stride():
            a, b = a.contiguous(), b.contiguous()
        keep += [a, b]
        pl += [plane(a), plane(b)]
    planes = (Plane * 6)(*pl)
    p = make_params(**kw)
    dev = keep[0].device
    n = ctypes.c_size_t()
    _check(lib.gbssim_video_workspace_size(planes, ctypes.byref(p), ctypes.byref(n)), "gbssim_video_workspace_size")
    ws = torch.empty(max(int(n.value), 1), dtype=torch.uint8, device=dev)
    frames = keep[0].shape[0]
    fr = torch.empty(frames, dtype=torch.float64, device=dev)
    ps = torch.empty((3, frames), dtype=torch.float64, device=dev)
    vid = torch.empty(3, dtype=torch.float64, device=dev)
    w = (ctypes.c_double * 3)(*[float(t) for t in weights])
    _check(lib.gbssim_video(planes, ctypes.byref(p), w, float(percentile), float(pp_r), fr.data_ptr(), ps.data_ptr(),
                            vid.data_ptr(), ws.data_ptr(), ws.numel(), _stream(dev)), "gbssim_video")
    return fr, ps, vid


class BatchPlan:
    """A ragged batch (gbssim_batch_plan): SSIM or MS-SSIM of pairs of mixed
    sizes in one persistent kernel launch.  ``xs``/``ys`` are lists of CUDA
    tensors (H, W) or (N, H, W) of one dtype; the plan is bound to these
    tensors (keep them alive; refill them in place to score new data).

    ``run()`` enqueues one run and returns the float64 scores (one per image,
    entries expanded in order).  ``capture()`` records one run into a CUDA
    graph; ``replay()`` launches it again.  Tuning knobs (0 = default):
    ``seg_rows`` output rows per work item, ``ctas_per_sm`` resident CTAs
    per SM, ``tile_w`` output columns per work item (32, 64 or 128; the CTA
    runs 4 x tile_w threads)."""

    def __init__(self, xs, ys, multiscale: bool = False, seg_rows: int = 0, ctas_per_sm: int = 0,
                 wait_limit: int = 0, flags: int = 0, tile_w: int = 0, **kw):
        if len(xs) != len(ys) or not xs:
            raise ValueError("xs and ys must be non-empty lists of equal length")
        self.xs = [_as_batch(t) for t in xs]
        self.ys = [_as_batch(t) for t in ys]
        self.device = self.xs[0].device
        if multiscale:
            kw.setdefault("exponents", MSSSIM_EXPONENTS[: kw.get("scales", 5)])
        self.params = make_params(**kw)
        self.multiscale = bool(multiscale)
        px = (Plane * len(xs))(*[plane(t) for t in self.xs])
        py = (Plane * len(ys))(*[plane(t) for t in self.ys])
        tun = Tuning(int(seg_rows), int(ctas_per_sm), int(wait_limit), int(flags), int(tile_w))
        self.tile_w = int(tile_w) or 64
        self._plan = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            _check(lib.gbssim_batch_plan(px, py, len(xs), ctypes.byref(self.params), int(self.multiscale),
                                         ctypes.byref(tun), ctypes.byref(self._plan)), "gbssim_batch_plan")
        n = ctypes.c_size_t()
        _check(lib.gbssim_batch_workspace_size(self._plan, ctypes.byref(n)), "gbssim_batch_workspace_size")
        self.ws = torch.empty(max(int(n.value), 1), dtype=torch.uint8, device=self.device)
        ni, items, grid, rows = (ctypes.c_int32() for _ in range(4))
        lib.gbssim_batch_info(self._plan, ctypes.byref(ni), ctypes.byref(items), ctypes.byref(grid), ctypes.byref(rows))
        self.n_images, self.total_items, self.grid, self.seg_rows = ni.value, items.value, grid.value, rows.value
        scales = self.params.scales if self.multiscale else 1
        self.scores = torch.empty(self.n_images, dtype=torch.float64, device=self.device)
        self.per_scale = torch.empty((self.n_images, scales, 2), dtype=torch.float64, device=self.device)
        self._status = torch.zeros(1, dtype=torch.int32, device=self.device)
        self.graph = None

    def run(self) -> torch.Tensor:
        _check(lib.gbssim_batch_run(self._plan, self.scores.data_ptr(), self.per_scale.data_ptr(),
                                    self.ws.data_ptr(), self.ws.numel(), _stream(self.device)),
               "gbssim_batch_run")
        return self.scores

    def status(self) -> int:
        """Status word of the last run (0, or ERR_TIMEOUT); synchronises."""
        _check(lib.gbssim_batch_status(self._plan, self.ws.data_ptr(), self._status.data_ptr(),
                                       _stream(self.device)), "gbssim_batch_status")
        return int(self._status.item())

    def capture(self):
        """Record one run into a CUDA graph (after one eager warm-up run)."""
        self.run()
        torch.cuda.synchronize(self.device)
        g = torch.cuda.CUDAGraph()
        s = torch.cuda.Stream(self.device)
        s.wait_stream(torch.cuda.current_stream(self.device))
        with torch.cuda.stream(s):
            with torch.cuda.graph(g, stream=s):
                self.run()
        torch.cuda.current_stream(self.device).wait_stream(s)
        self.graph = g
        return g

    def replay(self) -> torch.Tensor:
        if self.graph is None:
            self.capture()
        self.graph.replay()
        return self.scores

    def __del__(self):
        try:
            if self._plan:
                lib.gbssim_batch_free(self._plan)
                self._plan = ctypes.c_void_p()
        except Exception:
            pass
