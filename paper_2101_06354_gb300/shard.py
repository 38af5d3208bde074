"""Sharding SSIM work across ranks (one process per GPU).

SSIM and MS-SSIM scores of different pairs (or frames) are independent, so a
workload splits across ranks with no exchange on the data path: each rank
scores its own share on its own GPU, and only the per-pair scores (doubles)
are gathered afterwards.

* ``partition(sizes, world)``: deterministic longest-processing-time split of
  pairs by pixel count, so ranks get near-equal work.
* ``gather_scores(local, indices, n, group)``: all-gather of the per-rank
  scores back into input order (any torch.distributed backend; tests use
  gloo on CPU).
"""
from __future__ import annotations

import torch
import torch.distributed as dist


def partition(sizes, world: int):
    """Split pair indices over `world` ranks, balancing total pixels.

    sizes: list of (h, w).  Returns a list of `world` sorted index lists.
    Pairs are placed largest first on the currently least-loaded rank (ties
    to the lower rank), which keeps every rank within one pair of the mean."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(sizes)), key=lambda i: (-sizes[i][0] * sizes[i][1], i))
    loads = [0] * world
    parts = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda k: (loads[k], k))
        parts[r].append(i)
        loads[r] += sizes[i][0] * sizes[i][1]
    return [sorted(p) for p in parts]


def gather_scores(local: torch.Tensor, indices, n: int, group=None) -> torch.Tensor:
    """All-gather per-rank scores into one float64 CPU tensor of length n in
    input order.  `local[k]` is the score of pair `indices[k]`."""
    world = dist.get_world_size(group)
    local = local.detach().to("cpu", torch.float64).reshape(-1)
    idx = torch.as_tensor(list(indices), dtype=torch.int64)
    if local.numel() != idx.numel():
        raise ValueError("one score per index")
    counts = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(counts, torch.tensor([idx.numel()], dtype=torch.int64), group=group)
    m = int(max(c.item() for c in counts))
    pad_v = torch.zeros(m, dtype=torch.float64)
    pad_i = torch.full((m,), -1, dtype=torch.int64)
    pad_v[: local.numel()] = local
    pad_i[: idx.numel()] = idx
    vs = [torch.zeros(m, dtype=torch.float64) for _ in range(world)]
    is_ = [torch.zeros(m, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(vs, pad_v, group=group)
    dist.all_gather(is_, pad_i, group=group)
    out = torch.full((n,), float("nan"), dtype=torch.float64)
    for v, i in zip(vs, is_):
        keep = i >= 0
        out[i[keep]] = v[keep]
    return out
