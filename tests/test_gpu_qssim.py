"""gbssim_qssim (Section "Quaternion SSIM") against the FP64 oracle
(oracle/quaternion.py) through the C ABI: uint8 pictures (exact integer sums,
held to 1e-9), float pictures (fp32 / fp16 / bf16 storage, the oracle on the
same rounded values, the pooled bound 1e-6), odd sizes, row pitches wider
than the picture, a 4K pair, the closed forms, and the argument errors."""
import ctypes

import numpy as np
import pytest
import torch

from oracle import quaternion as Q

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


def _tri_pair(n, h, w, seed):
    """Three smooth-noise planes per picture; the distorted planes are the
    block-quantised, noisy versions (each plane from its own seeds)."""
    from paper_2101_06354_gb300 import synth

    xs, ys = [], []
    for c in range(3):
        x, y = synth.luma_pairs_u8(n, h, w, seed_ref=seed + 10 * c, seed_dist=seed + 10 * c + 500)
        xs.append(x)
        ys.append(y)
    return xs, ys


def _ref(xs, ys, i, scale=1.0, **kw):
    fx = [t[i].double().cpu().numpy() * scale for t in xs]
    fy = [t[i].double().cpu().numpy() * scale for t in ys]
    return Q.qssim_terms(fx, fy, **kw)


@pytest.mark.parametrize("n,h,w", [(3, 64, 80), (2, 97, 131), (1, 2, 2), (1, 2, 300), (2, 1081, 7)])
def test_qssim_u8_matches_oracle(g, n, h, w):
    xs, ys = _tri_pair(n, h, w, seed=h + w)
    score, terms = g.qssim([t.to(DEV) for t in xs], [t.to(DEV) for t in ys], return_terms=True)
    score, terms = score.cpu().numpy(), terms.cpu().numpy()
    for i in range(n):
        lum, cs, s = _ref(xs, ys, i)
        assert abs(score[i] - s) <= 1e-9, (i, score[i], s)
        assert abs(terms[i, 0] - lum) <= 1e-9 and abs(terms[i, 1] - cs) <= 1e-9


@pytest.mark.parametrize("dtype", [torch.float32, torch.float16, torch.bfloat16])
def test_qssim_float_matches_oracle_on_rounded_values(g, dtype):
    xs, ys = _tri_pair(2, 150, 171, seed=7)
    xf = [(t.float() / 255).to(dtype) for t in xs]
    yf = [(t.float() / 255).to(dtype) for t in ys]
    score, terms = g.qssim([t.to(DEV) for t in xf], [t.to(DEV) for t in yf], return_terms=True, L=1.0)
    for i in range(2):
        lum, cs, s = _ref(xf, yf, i, L=1.0)
        assert abs(score[i].item() - s) <= 1e-6
        assert abs(terms[i, 0].item() - lum) <= 1e-6 and abs(terms[i, 1].item() - cs) <= 1e-6


def test_qssim_strided_planes_and_constants(g):
    xs, ys = _tri_pair(2, 90, 120, seed=11)
    # a window of each plane: row pitch 120 > width 100
    xv = [t[:, :, 10:110].to(DEV) for t in xs]
    yv = [t[:, :, 10:110].to(DEV) for t in ys]
    px = (g.Plane * 3)(*[g.Plane(t.data_ptr(), g.U8, 2, 90, 100, t.stride(1), t.stride(0)) for t in xv])
    py = (g.Plane * 3)(*[g.Plane(t.data_ptr(), g.U8, 2, 90, 100, t.stride(1), t.stride(0)) for t in yv])
    p = g.make_params(K1=0.0, K2=0.0)  # the printed constant-free form
    nb = ctypes.c_size_t()
    assert g.lib.gbssim_qssim_workspace_size(ctypes.byref(px[0]), ctypes.byref(nb)) == 0
    ws = torch.empty(nb.value, dtype=torch.uint8, device=DEV)
    score = torch.empty(2, dtype=torch.float64, device=DEV)
    assert g.lib.gbssim_qssim(px, py, ctypes.byref(p), score.data_ptr(), None, ws.data_ptr(), ws.numel(),
                              torch.cuda.current_stream().cuda_stream) == 0
    for i in range(2):
        fx = [t[i, :, 10:110].double().numpy() for t in xs]
        fy = [t[i, :, 10:110].double().numpy() for t in ys]
        assert abs(score[i].item() - Q.qssim(fx, fy, K1=0.0, K2=0.0)) <= 1e-9


def test_qssim_closed_forms(g):
    xs, _ = _tri_pair(1, 40, 50, seed=5)
    d = [t.to(DEV) for t in xs]
    assert abs(g.qssim(d, d).item() - 1.0) <= 1e-12
    # constant colours: the DC term sqrt((2 a.b + C1)^2 + 4 |a x b|^2) / (|a|^2 + |b|^2 + C1)
    a, b = np.array([200.0, 10.0, 40.0]), np.array([180.0, 30.0, 45.0])
    ca = [torch.full((1, 8, 9), v, dtype=torch.uint8, device=DEV) for v in a]
    cb = [torch.full((1, 8, 9), v, dtype=torch.uint8, device=DEV) for v in b]
    C1 = (0.01 * 255) ** 2
    want = np.sqrt((2 * a @ b + C1) ** 2 + 4 * np.sum(np.cross(a, b) ** 2)) / (a @ a + b @ b + C1)
    assert abs(g.qssim(ca, cb).item() - want) <= 1e-12


def test_qssim_4k_pair(g):
    xs, ys = _tri_pair(2, 2160, 3840, seed=21)
    score = g.qssim([t.to(DEV) for t in xs], [t.to(DEV) for t in ys]).cpu().numpy()
    for i in range(2):
        assert abs(score[i] - _ref(xs, ys, i)[2]) <= 1e-9


def test_qssim_errors(g):
    x = torch.zeros((1, 1, 40), dtype=torch.uint8, device=DEV)
    with pytest.raises(g.GbssimError) as e:
        g.qssim([x, x, x], [x, x, x])
    assert e.value.status == g.ERR_TOO_SMALL
    a = torch.zeros((1, 8, 8), dtype=torch.uint8, device=DEV)
    b = torch.zeros((1, 8, 9), dtype=torch.uint8, device=DEV)
    with pytest.raises(g.GbssimError) as e:
        g.qssim([a, a, a], [a, b, a])
    assert e.value.status == g.ERR_INVALID_ARG
