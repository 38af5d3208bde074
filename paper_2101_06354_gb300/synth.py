"""Seeded synthetic image pairs with the structure of the paper's workloads.

This module is the only code shared by the CUDA path's tests/benchmark and the
CPU oracle.  It produces input bytes only and holds none of the SSIM
arithmetic.  The subjective databases the paper measures on (LIVE IQA, TID2013,
LIVE VQA, Netflix Public) are not available, so these fields stand in for them:

* smooth noise: N(0,1) white noise drawn from a seeded ``torch.Generator``
  (CPU), low-pass filtered by a sigma = 3 Gaussian truncated at +-12 taps
  (valid convolution of a field 24 px larger than the output, so no border
  rule is needed), then min-max rescaled to [0, 255];
* distortions: additive Gaussian noise, and 8x8 block-mean quantisation
  (each 8x8 block keeps its mean b; pixels become b + step*round((x-b)/step)),
  the blocking artefact of transform coding;
* rounding is half-to-even and uint8 values are clipped to [0, 255].

Every generator takes explicit seeds and an optional device on which the
filtering runs (the random draws are always made on the CPU generator, so the
same seed gives the same field on any device up to the filter's rounding).
"""
from __future__ import annotations

import math

import torch
import torch.nn.functional as F

_BLUR_SIGMA = 3.0
_BLUR_RADIUS = 12


def _normal(shape, seed: int) -> torch.Tensor:
    g = torch.Generator().manual_seed(int(seed))
    return torch.randn(*shape, generator=g, dtype=torch.float32)


def _blur_taps(device) -> torch.Tensor:
    t = torch.arange(-_BLUR_RADIUS, _BLUR_RADIUS + 1, dtype=torch.float64)
    g = torch.exp(-(t * t) / (2 * _BLUR_SIGMA ** 2))
    return (g / g.sum()).to(torch.float32).to(device)


def smooth_noise(h: int, w: int, seed: int, device="cpu", n: int = 1) -> torch.Tensor:
    """``n`` smooth-noise fields of size h x w as float32 in [0, 255]
    (shape (n, h, w)); field i uses seed ``seed + i``."""
    r = _BLUR_RADIUS
    out = torch.empty((n, h, w), dtype=torch.float32, device=device)
    taps = _blur_taps(device)
    for i in range(n):
        z = _normal((h + 2 * r, w + 2 * r), seed + i).to(device)
        z = F.conv2d(z[None, None], taps.view(1, 1, 1, -1))
        z = F.conv2d(z, taps.view(1, 1, -1, 1))[0, 0]
        lo, hi = z.min(), z.max()
        out[i] = (z - lo) * (255.0 / (hi - lo))
    return out


def to_u8(v: torch.Tensor) -> torch.Tensor:
    """Round half-to-even and clip to [0, 255]."""
    return torch.clamp(torch.round(v), 0, 255).to(torch.uint8)


def add_noise(x: torch.Tensor, sigma: float, seed: int) -> torch.Tensor:
    """x + N(0, sigma^2) (float32)."""
    return x.to(torch.float32) + sigma * _normal(tuple(x.shape), seed).to(x.device)


def block_quantise(x: torch.Tensor, step, block: int = 8) -> torch.Tensor:
    """8x8 block-mean quantisation of a (..., H, W) float field.  Pixels of
    incomplete edge blocks use the mean of the pixels that exist.  ``step`` is a
    scalar or a tensor broadcastable over the leading dimensions."""
    x = x.to(torch.float32)
    H, W = x.shape[-2:]
    hb, wb = math.ceil(H / block), math.ceil(W / block)
    pad = (0, wb * block - W, 0, hb * block - H)
    lead = x.shape[:-2]
    xf = x.reshape(-1, 1, H, W)
    ones = torch.ones_like(xf)
    s = F.avg_pool2d(F.pad(xf, pad), block, divisor_override=1)
    c = F.avg_pool2d(F.pad(ones, pad), block, divisor_override=1)
    b = (s / c).repeat_interleave(block, -2).repeat_interleave(block, -1)[..., :H, :W]
    b = b.reshape(*lead, H, W)
    step = torch.as_tensor(step, dtype=torch.float32, device=x.device)
    while step.dim() < x.dim():
        step = step.unsqueeze(-1)
    return b + step * torch.round((x - b) / step)


def single_pair_u8(h: int = 256, w: int = 256, seed_ref: int = 1, seed_noise: int = 2,
                   noise_sigma: float = 10.0, device="cpu"):
    """Reference = smooth noise; distorted = reference + N(0, noise_sigma^2),
    rounded and clipped (the 256x256 single-pair workload)."""
    x = smooth_noise(h, w, seed_ref, device)[0]
    y = add_noise(x, noise_sigma, seed_noise)
    return to_u8(x), to_u8(y)


def luma_pairs_u8(n: int, h: int = 1080, w: int = 1920, seed_ref: int = 10,
                  seed_dist: int = 1000, step: float = 12.0, noise_sigma: float = 4.0,
                  device="cpu"):
    """n uint8 pairs (n, h, w): smooth-noise references (seeds seed_ref+i) and
    distorted = block quantisation to ``step`` plus N(0, noise_sigma^2) noise
    (seeds seed_dist+i), rounded and clipped (the 1080p MS-SSIM workload)."""
    x = smooth_noise(h, w, seed_ref, device, n)
    y = block_quantise(x, step)
    for i in range(n):
        y[i] = add_noise(y[i], noise_sigma, seed_dist + i)
    return to_u8(x), to_u8(y)


def video_yuv420_u8(frames: int, h: int = 2160, w: int = 3840, drift: int = 2,
                    seeds=(20, 21, 22), device="cpu"):
    """Temporally correlated YUV 4:2:0 video pairs.

    Each plane is a crop of one smooth-noise canvas that drifts ``drift`` px
    per frame (luma) and drift/2 px (chroma); the distortion of frame t is
    8x8 block quantisation with step round(4 + 20 t/(frames-1)).  Returns
    dict plane -> (ref, dist) uint8 tensors of shape (frames, h_p, w_p)."""
    out = {}
    steps = torch.tensor([round(4 + 20 * t / max(frames - 1, 1)) for t in range(frames)],
                         dtype=torch.float32, device=device)
    for name, (ph, pw, d, sd) in {"y": (h, w, drift, seeds[0]),
                                  "u": (h // 2, w // 2, max(drift // 2, 1), seeds[1]),
                                  "v": (h // 2, w // 2, max(drift // 2, 1), seeds[2])}.items():
        canvas = smooth_noise(ph, pw + d * (frames - 1), sd, device)[0]
        ref = torch.stack([canvas[:, d * t: d * t + pw] for t in range(frames)])
        dist = block_quantise(ref, steps)
        out[name] = (to_u8(ref), to_u8(dist))
    return out


RAGGED_SIZES = ((640, 360), (854, 480), (1280, 720), (1920, 1080), (2560, 1440), (3840, 2160))


def ragged_sizes(n_regular: int = 512, n_odd: int = 64, seed_regular: int = 30,
                 seed_odd: int = 31):
    """(h, w) list: n_regular sizes drawn uniformly from the six standard
    resolutions, then n_odd sizes with W ~ U[177, 3840], H ~ U[177, 2160],
    both forced odd."""
    g = torch.Generator().manual_seed(seed_regular)
    idx = torch.randint(0, len(RAGGED_SIZES), (n_regular,), generator=g).tolist()
    sizes = [(RAGGED_SIZES[i][1], RAGGED_SIZES[i][0]) for i in idx]
    g2 = torch.Generator().manual_seed(seed_odd)
    ws = torch.randint(177, 3841, (n_odd,), generator=g2).tolist()
    hs = torch.randint(177, 2161, (n_odd,), generator=g2).tolist()
    sizes += [(h | 1, w | 1) for h, w in zip(hs, ws)]
    return sizes


def ragged_pairs_u8(sizes, seed_ref: int = 10, seed_dist: int = 1000, device="cpu"):
    """One uint8 pair per (h, w) in ``sizes``, content as luma_pairs_u8."""
    xs, ys = [], []
    for i, (h, w) in enumerate(sizes):
        x, y = luma_pairs_u8(1, h, w, seed_ref + i, seed_dist + i, device=device)
        xs.append(x[0])
        ys.append(y[0])
    return xs, ys


def loss_pairs_float(b: int = 32, c: int = 3, h: int = 512, w: int = 512, seed_ref: int = 40,
                     seed_noise: int = 41, noise_sigma: float = 0.05, device="cpu"):
    """Float pairs in [0, 1] (shape (b, c, h, w)): smooth noise / 255 and
    reference + N(0, noise_sigma^2), not clipped (the loss workload)."""
    x = smooth_noise(h, w, seed_ref, device, b * c).reshape(b, c, h, w) / 255.0
    y = add_noise(x, noise_sigma, seed_noise)
    return x, y
