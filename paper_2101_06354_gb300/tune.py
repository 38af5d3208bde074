"""Autotuner for the ragged persistent batch (gbssim_batch_*).

Times candidate tunings of one batch -- the work-item shape (output rows per
item and the strip width, i.e. output columns per item, which sets the
threads per CTA at 4 x the width) and the resident CTAs per SM -- with CUDA
events on the current stream and keeps the fastest.  Results
are cached in a JSON file keyed by GPU name, dtype, MS-SSIM flag and a size
class of the batch (the image sizes rounded to powers of two and their
counts), so later plans of a similar batch skip the search.  The cache lives
at $GBSSIM_TUNE_CACHE, else ~/.cache/gbssim/tune.json; a missing or unreadable
cache is rebuilt.
"""
from __future__ import annotations

import json
import math
import os
from collections import Counter

import torch

from . import gbssim

# (seg_rows, ctas_per_sm, tile_w): 0 CTAs = as many as fit; the narrow strips
# (128 threads a CTA) also try half residency, the wide ones (512 threads)
# fit one CTA an SM
CANDIDATES = [(rows, ctas, tw) for tw, ctas_list in ((32, (0, 4)), (64, (0, 2)), (128, (0,)))
              for rows in (64, 128, 256, 512, 1024, 2048) for ctas in ctas_list]


def cache_path() -> str:
    return os.environ.get("GBSSIM_TUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "gbssim", "tune.json"))


def _load():
    try:
        with open(cache_path()) as f:
            d = json.load(f)
        return d if isinstance(d, dict) else {}
    except Exception:
        return {}


def _store(d):
    path = cache_path()
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = path + ".tmp"
        with open(tmp, "w") as f:
            json.dump(d, f, indent=1, sort_keys=True)
        os.replace(tmp, path)
    except OSError:
        pass


def signature(xs, multiscale: bool) -> str:
    """GPU, dtype, mode and the size classes of the batch."""
    classes = Counter()
    for t in xs:
        b = gbssim._as_batch(t)
        h, w = b.shape[1], b.shape[2]
        classes["%dx%d" % (2 ** round(math.log2(h)), 2 ** round(math.log2(w)))] += b.shape[0]
    name = torch.cuda.get_device_name(xs[0].device)
    parts = ",".join("%s:%d" % kv for kv in sorted(classes.items()))
    return "%s|%s|%s|%s" % (name, str(xs[0].dtype).replace("torch.", ""), "ms" if multiscale else "ss", parts)


def time_plan(plan: "gbssim.BatchPlan", reps: int = 5) -> float:
    """Median milliseconds of `reps` runs (after one warm-up)."""
    plan.run()
    stream = torch.cuda.current_stream(plan.device)
    times = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        plan.run()
        b.record(stream)
        b.synchronize()
        times.append(a.elapsed_time(b))
    return sorted(times)[len(times) // 2]


def tune(xs, ys, multiscale: bool = False, candidates=None, reps: int = 5, use_cache: bool = True, **kw):
    """Return (seg_rows, ctas_per_sm, tile_w, results) for this batch;
    candidates are (seg_rows, ctas_per_sm[, tile_w]) tuples (tile_w 64 when
    left out); results maps each tried candidate "rows/ctas/tile_w" to its
    median milliseconds."""
    key = signature(xs, multiscale)
    cache = _load() if use_cache else {}
    if use_cache and key in cache:
        c = cache[key]
        return c["seg_rows"], c["ctas_per_sm"], c.get("tile_w", 64), c.get("results", {})
    results = {}
    best = None
    for cand in (candidates or CANDIDATES):
        rows, ctas, tw = (tuple(cand) + (64,))[:3]
        plan = gbssim.BatchPlan(xs, ys, multiscale=multiscale, seg_rows=rows, ctas_per_sm=ctas, tile_w=tw, **kw)
        ms = time_plan(plan, reps)
        results["%d/%d/%d" % (rows, ctas, tw)] = ms
        if best is None or ms < best[0]:
            best = (ms, rows, ctas, tw)
        del plan
    cache[key] = {"seg_rows": best[1], "ctas_per_sm": best[2], "tile_w": best[3], "ms": best[0],
                  "results": results}
    if use_cache:
        _store(cache)
    return best[1], best[2], best[3], results


def autotuned_plan(xs, ys, multiscale: bool = False, **kw) -> "gbssim.BatchPlan":
    """A BatchPlan with the tuned (or cached) knobs for this batch."""
    rows, ctas, tw, _ = tune(xs, ys, multiscale, **kw)
    return gbssim.BatchPlan(xs, ys, multiscale=multiscale, seg_rows=rows, ctas_per_sm=ctas, tile_w=tw, **kw)
