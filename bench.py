"""Benchmark: 1080p MS-SSIM throughput (Mpx-pairs/s) on GB300.

Workload (one "step"): MS-SSIM of 64 uint8 luma pairs of 1920x1080 (smooth
noise references, block-quantised + noisy distortions), 5 scales, 11x11
Gaussian sigma = 1.5, 2x2 average pyramid, exponents 0.0448/0.2856/0.3001/
0.2363/0.1333, all through the C ABI (gbssim_msssim).  Inputs (265 MB) are
larger than L2, so no flush is needed between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gbssim|reference]

N > 1 runs under torchrun, one rank per GPU, each rank on its own 64 pairs
(weak scaling, no data-path collective); rank 0 prints one JSON line.
--impl reference times the FP64 CPU oracle on a bounded sample of the same
workload on the host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_PAIRS, H, W = 64, 1080, 1920
PX_PER_PAIR = H * W
METRIC = "1080p MS-SSIM Mpx-pairs/s (% HBM roofline); SSIM-loss fwd+bwd Mpx/s"
UNIT = "Mpx-pairs/s"
WORKLOAD = "msssim_1080p_u8_x64"
CONFIG = {"workload": WORKLOAD, "pairs_per_gpu": N_PAIRS, "height": H, "width": W, "dtype_in": "u8",
          "scales": 5, "window": "gaussian11_sigma1.5", "l2": "inputs (265 MB) larger than L2, no flush"}
# FP32 non-tensor peak derived from the unit counts (152 SMs x 128 FP32 lanes
# x 2 flop (FMA) x 2.070 GHz max SM clock); the roofline uses the rate the
# FMA probe measures on the GPU at hand, this figure is reported beside it
FP32_PEAK_DERIVED_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12
# algorithmic FLOP per SSIM output: 5 moments x 2 separable passes x 11 taps x 2 + 3 products + ~17 formula
FLOP_PER_OUTPUT = 240
# MS-SSIM pools only mean cs below the last level: those outputs need no
# luminance term (2 mu_x mu_y + C1, mu_x^2 + mu_y^2 + C1, the divide and the
# product l * cs: 6 FLOP)
FLOP_PER_CS_OUTPUT = 234
# pyramid levels of the workload (floor halving)
LEVELS = [(H >> j, W >> j) for j in range(5)]
# kernels of libgbssim per MS-SSIM step: the persistent level kernel and the finaliser
LAUNCHES_PER_STEP = 2
# chunks of the end-to-end step's host pipeline; 0 streams (one launch over all
# pairs, each copy group scored as soon as its arrival flag is set)
E2E_CHUNKS = 0
# DRAM bytes (read + write) of one persistent launch on this workload, from an
# ncu capture of dram__bytes_read.sum + dram__bytes_write.sum; valid only for
# the sources it was taken on (the kernel and the host code that sets its
# work items; sha256 of the files below, first 16 hex).
TRAFFIC = {"bytes": 429.174e6 + 158.580e6, "sources_sha": "a56ce214640a9ff6"}
TRAFFIC_SOURCES = ("paper_2101_06354_gb300/csrc/k_gauss.cu", "paper_2101_06354_gb300/csrc/api.cu")


def _sources_sha():
    import hashlib

    h = hashlib.sha256()
    for f in TRAFFIC_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _traffic():
    if TRAFFIC["bytes"] is None or TRAFFIC["sources_sha"] != _sources_sha():
        return None
    return TRAFFIC["bytes"]


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def measure_fp32_peak(gbssim, dev, iters: int = 4000):
    """FP32 FMA rate of this GPU (TFLOP/s): gbssim_fp32_probe, scalar FFMA
    and packed FFMA2 chains on 16 CTAs x 256 threads per SM, median of 5
    launches each (CUDA events on the launching stream); the larger of the
    two rates is the peak."""
    import torch

    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    blocks = 16 * sms
    sink = torch.empty(blocks * 256, device=dev)
    st = torch.cuda.current_stream(dev)
    rates = {}
    for packed in (0, 1):
        for _ in range(2):
            gbssim._check(gbssim.lib.gbssim_fp32_probe(packed, blocks, iters, sink.data_ptr(), st.cuda_stream),
                          "gbssim_fp32_probe")
        ts = []
        for _ in range(5):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            gbssim.lib.gbssim_fp32_probe(packed, blocks, iters, sink.data_ptr(), st.cuda_stream)
            e1.record(st)
            torch.cuda.synchronize(dev)
            ts.append(e0.elapsed_time(e1))
        ms = statistics.median(ts)
        rates["ffma2" if packed else "ffma"] = blocks * 256 * 512 * iters / (ms / 1e3) / 1e12
    return max(rates.values()), rates


def c1_latency(gbssim, synth, dev, samples: int = 5, back_to_back: int = 200):
    """Single 256x256 uint8 pair, SSIM with the 11x11 Gaussian (the smallest
    workload, latency-bound): per-call latency in microseconds, CUDA events
    around one gbssim_ssim_map call (+ its pooling finaliser) with L2 flushed
    (a 256 MB write) before each sample, median of 5; plus the L2-warm
    back-to-back rate."""
    import torch

    x, y = synth.single_pair_u8(256, 256, device="cpu")
    x, y = x.reshape(1, 256, 256).to(dev), y.reshape(1, 256, 256).to(dev)
    p = gbssim.make_params()
    wsc = gbssim.workspace(gbssim.plane(x), p, gbssim.OP_SSIM, dev)
    fn = lambda: gbssim.ssim(x, y, ws=wsc)
    for _ in range(5):
        fn()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    st = torch.cuda.current_stream(dev)
    lat = []
    for _ in range(samples):
        flush.fill_(1)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        fn()
        e1.record(st)
        torch.cuda.synchronize(dev)
        lat.append(e0.elapsed_time(e1) * 1e3)
    del flush
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(back_to_back):
        fn()
    e1.record(st)
    torch.cuda.synchronize(dev)
    b2b = e0.elapsed_time(e1) * 1e3 / back_to_back
    return {"latency_us": statistics.median(lat), "samples_us": lat, "back_to_back_us": b2b,
            "mpx_pairs_per_s_back_to_back": 256 * 256 / b2b, "kernels_per_call": 2,
            "config": "1 pair 256x256 u8, Gaussian 11 / 1.5, valid, K = 0.01 / 0.03, L = 255, FP64 pooled; "
                      "L2 flushed (256 MB write) before each latency sample"}


class ClockSampler:
    """nvidia-smi clock / throttle sampling in the background: every sample is
    stamped on arrival, so the summary can cover the whole timed phase or
    one window of it."""

    Q = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.lines = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "20"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        import datetime

        for line in self.proc.stdout:
            line = line.strip()
            try:  # nvidia-smi's own stamp (local time, ms): immune to pipe buffering
                ts = datetime.datetime.strptime(line.split(",")[0].strip(), "%Y/%m/%d %H:%M:%S.%f").timestamp()
            except ValueError:
                ts = time.time()
            self.lines.append((ts, line))

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self, t_begin: float = None, t_end: float = None):
        """Median SM clock, maximum clock and active throttle reasons of the
        samples stamped inside [t_begin, t_end] (time.time() seconds; all
        samples by default)."""
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ts, ln in self.lines:
            if (t_begin is not None and ts < t_begin) or (t_end is not None and ts > t_end):
                continue
            f = [t.strip() for t in ln.split(",")][1:]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def run_reference(args):
    """The FP64 CPU oracle on a bounded sample (a few 1080p pairs per step)."""
    ws, rank, _ = _dist()
    if rank != 0:
        return
    import numpy as np

    import oracle
    from paper_2101_06354_gb300 import synth

    sample = 4
    x, y = synth.luma_pairs_u8(sample, H, W)
    xs, ys = x.numpy(), y.numpy()
    step = lambda: [oracle.msssim(xs[i], ys[i], mode="separable") for i in range(sample)]
    for _ in range(args.warmup):
        step()
    t = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = time.perf_counter() - t
    value = sample * PX_PER_PAIR * args.steps / dt / 1e6
    cores = oracle.num_threads()
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": dict(CONFIG, sample_pairs_per_step=sample), "impl": "reference",
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "%d of the 64 1080p pairs per step, FP64 oracle, separable mode "
                                       "(row then column passes), OpenMP over rows" % sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def _oracle_rate(oracle, xs, ys, min_seconds: float, max_passes: int = 16):
    """Passes of the separable FP64 oracle over the sample pairs until about
    min_seconds; returns (Mpx-pairs/s, passes, seconds)."""
    passes = 0
    t = time.perf_counter()
    while passes < max_passes and (passes == 0 or time.perf_counter() - t < min_seconds):
        for i in range(len(xs)):
            oracle.msssim(xs[i], ys[i], mode="separable")
        passes += 1
    dt = time.perf_counter() - t
    return passes * len(xs) * PX_PER_PAIR / dt / 1e6, passes, dt


def cpu_baseline(min_seconds: float = 6.0):
    """The FP64 oracle (its separable mode: a row pass then a column pass per
    window statistic, the plain CPU implementation of the definition) timed on
    all host cores and on one core, on bounded samples of the 64 pairs:
    16 pairs on all cores, 2 pairs on one core, passes repeated until about
    min_seconds each."""
    import oracle
    from paper_2101_06354_gb300 import synth

    x, y = synth.luma_pairs_u8(16, H, W)
    xs, ys = x.numpy(), y.numpy()
    cores = oracle.num_threads()
    v_all, p_all, t_all = _oracle_rate(oracle, xs, ys, min_seconds)
    oracle.set_num_threads(1)
    try:
        v_one, p_one, t_one = _oracle_rate(oracle, xs[:2], ys[:2], min_seconds)
    finally:
        oracle.set_num_threads(cores)
    return {"value": v_all, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "%d passes over 16 of the 64 1080p pairs, MS-SSIM, FP64 oracle in its separable mode "
                      "(row then column passes), all %d host cores (OpenMP, %.1f s)" % (p_all, cores, t_all),
            "single_core": {"value": v_one, "unit": UNIT, "cores": 1,
                            "sample": "%d passes over 2 of the pairs on one core (%.1f s)" % (p_one, t_one)}}


def _rate(fn, units: float, min_seconds: float, max_passes: int = 10000):
    """Calls of fn until about min_seconds; returns (units per second / 1e6, passes, seconds)."""
    passes = 0
    t = time.perf_counter()
    while passes < max_passes and (passes == 0 or time.perf_counter() - t < min_seconds):
        fn()
        passes += 1
    dt = time.perf_counter() - t
    return passes * units / dt / 1e6, passes, dt


def oracle_workloads(min_seconds: float = 1.5):
    """The FP64 oracle on bounded samples of the secondary workloads, on all
    host cores and on one core: a 256x256 pair (SSIM, the latency case); two
    frames of the 3840x2160 YUV 4:2:0 video (SSIM per plane); four pairs of
    the ragged batch (MS-SSIM); one 512x512 plane of the loss batch (SSIM and
    its gradient w.r.t. y, L = 1).  Gaussian windows use the oracle's
    separable window statistics; the gradient is its direct form."""
    import oracle
    from paper_2101_06354_gb300 import synth

    taps = oracle.taps_1d("gaussian", 11)

    def ssim_sep(a, b, L=255.0):
        st = oracle.window_stats_separable(a, b, taps)
        C1, C2 = oracle.constants(L=L)
        return oracle.mean(oracle.ssim_terms(st, C1, C2)[2])

    c1x, c1y = synth.luma_pairs_u8(1, 256, 256)
    c1x, c1y = c1x[0].numpy(), c1y[0].numpy()
    v = synth.video_yuv420_u8(2, 2160, 3840)
    planes = [(v[p][0][i].numpy(), v[p][1][i].numpy()) for i in range(2) for p in "yuv"]
    vpx = sum(a.size for a, _ in planes)
    sizes = synth.ragged_sizes(512, 64)[:4]
    rx, ry = synth.ragged_pairs_u8(sizes)
    rx, ry = [t.numpy() for t in rx], [t.numpy() for t in ry]
    lx, ly = synth.loss_pairs_float(1, 1, 512, 512)
    lx, ly = lx[0, 0].double().numpy(), ly[0, 0].double().numpy()

    def loss_step():
        ssim_sep(lx, ly, L=1.0)
        oracle.ssim_grad(lx, ly, L=1.0)

    work = {
        "c1_256": (lambda: ssim_sep(c1x, c1y), 256 * 256, UNIT, "1 pair 256x256 u8, SSIM"),
        "video_yuv420_4k": (lambda: [ssim_sep(a, b) for a, b in planes], vpx, UNIT,
                            "2 of the 120 frames 3840x2160 YUV 4:2:0, SSIM per plane"),
        "ragged_msssim": (lambda: [oracle.msssim(a, b, mode="separable") for a, b in zip(rx, ry)],
                          sum(h * w for h, w in sizes), UNIT,
                          "4 of the 576 ragged pairs (%s), MS-SSIM" % ", ".join("%dx%d" % (w, h) for h, w in sizes)),
        "loss_fwd_bwd": (loss_step, 512 * 512, "Mpx/s", "1 plane 512x512 of the 32x3 loss batch, SSIM + gradient"),
    }
    cores = oracle.num_threads()
    out = {}
    for key, (fn, units, unit, sample) in work.items():
        va, pa, ta = _rate(fn, units, min_seconds)
        oracle.set_num_threads(1)
        try:
            v1, p1, t1 = _rate(fn, units, min_seconds)
        finally:
            oracle.set_num_threads(cores)
        out[key] = {"unit": unit, "all_cores": va, "cores": cores, "single_core": v1,
                    "sample": "%s; %d passes on all cores (%.1f s), %d on one (%.1f s)" % (sample, pa, ta, p1, t1)}
    return out


def run_extras(args, gbssim, synth, x, y, dev, timed, ws):
    """Secondary figures on the same GPU: the 8x8 stride-4 integer box SSIM on
    the same 64 pairs (the HBM-bound path), and the SSIM-loss forward+backward
    of 32x3x512x512 float inputs in [0, 1] (fp32 and bf16 storage)."""
    import torch

    out = {}
    k_steps = max(10, args.steps // 5)
    k_short = max(100, args.steps)  # calls of well under 0.1 ms: enough of them for a steady-state figure
    hbm_peak, _ = _peaks()
    pb = gbssim.make_params(window="box", k=8, stride=4)
    wsb = gbssim.workspace(gbssim.plane(x), pb, gbssim.OP_SSIM, dev)
    box = lambda: gbssim.ssim(x, y, ws=wsb, window="box", k=8, stride=4)
    for _ in range(3):
        box()
    ms = timed(box, k_short) / k_short
    in_bytes = 2 * N_PAIRS * PX_PER_PAIR
    out["box8_s4"] = {"value": ws * N_PAIRS * PX_PER_PAIR / (ms / 1e3) / 1e6, "unit": UNIT, "ms_per_step": ms,
                      "hbm_gbs": in_bytes / (ms / 1e3) / 1e9, "hbm_frac": in_bytes / (ms / 1e3) / 1e9 / hbm_peak,
                      "config": "same 64 pairs, box 8x8 stride 4, exact int sums (column-walk kernel)"}
    # Enhanced SSIM on the same pairs: 4 x 4 block-mean downscaling (the
    # round-min rule at 1080p), 11 x 11 rectangular windows at stride 5, CoV
    # pooling -- three library calls per step
    enh = lambda: gbssim.enhanced_ssim(x, y)
    for _ in range(3):
        enh()
    ms = timed(enh, k_steps) / k_steps
    out["enhanced_ssim"] = {"value": ws * N_PAIRS * PX_PER_PAIR / (ms / 1e3) / 1e6, "unit": UNIT, "ms_per_step": ms,
                            "config": "same 64 pairs, z = 4 block means, box 11 stride 5, CoV pooling"}
    # pooling family on the 64 stored SSIM maps (1070 x 1910 floats each):
    # time per call and the bandwidth of the map passes each kind makes
    _, qmap = gbssim.ssim(x, y, return_map=True)
    nq, hq, wq = qmap.shape
    pq = gbssim.Plane(qmap.data_ptr(), gbssim.F32, nq, hq, wq, qmap.stride(1), qmap.stride(0))
    wsq = gbssim.workspace(pq, gbssim.Params(), gbssim.OP_POOL, dev)
    map_bytes = qmap.numel() * 4
    pool_res = {}
    # map passes: order statistics read the map three times on their value-bin
    # path (min / max, bin counts, the wanted bins' values; the radix passes
    # that would follow for a crowded map are not taken on these maps); PP
    # adds its moment pass
    for kind, pargs, passes in (("mean", (), 1), ("cov", (), 2), ("minkowski", (4.0,), 1), ("fns", (), 3),
                                ("pp", (6.0, 4000.0), 4)):
        fpool = lambda: gbssim.ssim_pool(qmap, kind, *pargs, ws=wsq)
        for _ in range(3):
            fpool()
        tq = timed(fpool, k_steps) / k_steps
        gbs = passes * map_bytes / (tq / 1e3) / 1e9
        pool_res[kind] = {"ms": tq, "map_passes": passes, "gbs": gbs, "hbm_frac": gbs / hbm_peak}
    out["pool_maps"] = dict(pool_res, config="64 SSIM maps 1070x1910 fp32 (523 MB), one double per map")
    del qmap
    # SSIM / MS-SSIM loss forward + backward, 32x3x512x512 in [0, 1] (L = 1),
    # fp32 and bf16 storage, both forms of the autograd Function:
    # "recompute" (the default: the backward recomputes the window moments)
    # and "stored" (the forward keeps the coefficient maps).  Algorithmic FLOP
    # per pixel and level: forward 240 (as the headline), coefficient pass 260
    # (forward + the three coefficient formulas), gradient pass 138 (three
    # maps x 11 taps x 2 passes x 2 + the combination); recompute = 240 + 260
    # + 138, stored = 260 + 138; MS-SSIM levels add a third.
    lx, ly = synth.loss_pairs_float(32, 3, 512, 512)
    px_step = 32 * 3 * 512 * 512
    flop_px = {"recompute": 240 + 260 + 138, "stored": 260 + 138}
    ms_px = sum((512 >> j) ** 2 for j in range(5)) / 512 ** 2  # pyramid pixels per input pixel
    loss_res = {}
    for name, dt in (("fp32", torch.float32), ("bf16", torch.bfloat16)):
        xd = lx.to(dev, dt)
        yd = ly.to(dev, dt).requires_grad_(True)
        esz = 4 if dt == torch.float32 else 2
        for ms_flag in (False, True):
            for form in ("recompute", "stored"):
                lf = gbssim.SSIMLoss(multiscale=ms_flag, recompute=form == "recompute", L=1.0)

                def fb():
                    yd.grad = None
                    loss = lf(xd, yd)
                    loss.backward()
                    return loss

                for _ in range(3):
                    fb()
                kk = max(5, args.steps // 20)
                t = timed(fb, kk) / kk
                flop = flop_px[form] * px_step * (ms_px if ms_flag else 1.0)
                key = ("msssim_" if ms_flag else "ssim_") + name + ("" if form == "recompute" else "_stored")
                loss_res[key] = {"value": ws * px_step / (t / 1e3) / 1e6, "unit": "Mpx/s", "ms_per_step": t,
                                 "form": form,
                                 "roofline": {"bound": "alu", "achieved": flop / (t / 1e3) / 1e12,
                                              "peak": args.fp32_peak, "unit": "TFLOP/s",
                                              "frac": flop / (t / 1e3) / 1e12 / args.fp32_peak,
                                              "flop_per_px": flop_px[form] * (ms_px if ms_flag else 1.0)},
                                 "hbm_frac": 3 * esz * px_step / (t / 1e3) / 1e9 / hbm_peak}
        del xd, yd
    out["loss_fwd_bwd"] = dict(loss_res, config="32x3x512x512, L=1, loss = 1 - mean score, grad w.r.t. y; "
                                                "default form recomputes the moments in the backward, *_stored "
                                                "keeps the forward's coefficient maps",
                               headline=loss_res["ssim_fp32"]["value"])

    # ragged batch: 512 pairs drawn from six resolutions 640x360..3840x2160 plus
    # 64 odd sizes, one persistent launch per run, replayed from a CUDA graph
    from paper_2101_06354_gb300 import tune

    sizes = synth.ragged_sizes(512, 64)
    xs, ys = synth.ragged_pairs_u8(sizes, device=dev)
    px_total = sum(h * w for h, w in sizes)
    rb = {"pairs": len(sizes), "mpx_pairs": px_total / 1e6}
    for name, msf in (("ssim", False), ("msssim", True)):
        rows, ctas, tw, _ = tune.tune(xs, ys, multiscale=msf, reps=2)
        plan = gbssim.BatchPlan(xs, ys, multiscale=msf, seg_rows=rows, ctas_per_sm=ctas, tile_w=tw)
        plan.capture()
        kk = max(3, args.steps // 50)
        t = timed(plan.replay, kk) / kk
        rb[name] = {"value": ws * px_total / (t / 1e3) / 1e6, "unit": UNIT, "ms_per_run": t,
                    "seg_rows": rows, "ctas_per_sm": ctas, "tile_w": tw, "grid": plan.grid,
                    "items": plan.total_items,
                    "status": plan.status()}
        del plan
    out["ragged_batch"] = rb
    del xs, ys

    # video: 120 frames of 3840x2160 YUV 4:2:0, per-plane SSIM, 6:1:1 colour
    # weights, temporal mean / 10th percentile / percentile pooling
    v = synth.video_yuv420_u8(120, 2160, 3840, device=dev)
    vx = [v[p][0] for p in "yuv"]
    vy = [v[p][1] for p in "yuv"]
    gbssim.video_ssim(vx, vy)
    kk = max(3, args.steps // 100)
    t = timed(lambda: gbssim.video_ssim(vx, vy), kk) / kk
    vpx = 120 * (3840 * 2160 + 2 * 1920 * 1080)
    fr, ps, vid = gbssim.video_ssim(vx, vy)
    out["video_yuv420_4k"] = {"value": ws * vpx / (t / 1e3) / 1e6, "unit": UNIT, "ms_per_video": t,
                              "frames": 120, "mean": vid[0].item(), "p10": vid[1].item(), "pp": vid[2].item()}
    # SSIM-3D (11 x 11 x 5 rectangular windows, exact integer sums) on the
    # 120 luma frames of the same video
    v3x, v3y = vx[0].contiguous(), vy[0].contiguous()
    fn3 = lambda: gbssim.ssim3d(v3x, v3y, kt=5, k=11)
    fn3()
    t3 = timed(fn3, kk) / kk
    px3 = 120 * 3840 * 2160
    s3, _ = fn3()
    out["ssim3d_4k_y"] = {"value": ws * px3 / (t3 / 1e3) / 1e6, "unit": UNIT, "ms_per_video": t3, "frames": 120,
                          "kt": 5, "k": 11, "hbm_gbs": 2 * px3 / (t3 / 1e3) / 1e9,
                          "hbm_frac": 2 * px3 / (t3 / 1e3) / 1e9 / hbm_peak, "score": s3.item()}
    # MS-SSIM-3D: the same windows on the 5 levels of each frame's pyramid
    fn4 = lambda: gbssim.msssim3d(v3x, v3y, kt=5, k=11, scales=5)
    fn4()
    t4 = timed(fn4, kk) / kk
    s4, _ = fn4()
    out["msssim3d_4k_y"] = {"value": ws * px3 / (t4 / 1e3) / 1e6, "unit": UNIT, "ms_per_video": t4, "frames": 120,
                            "kt": 5, "k": 11, "scales": 5, "score": s4.item()}
    del v, vx, vy
    return out


def run_gbssim(args):
    import torch
    import torch.distributed as dist

    from paper_2101_06354_gb300 import build

    build.build()
    from paper_2101_06354_gb300 import gbssim, synth

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if ws > 1:
            dist.barrier()

    # rank r processes its own 64 pairs (seeds offset by rank); generated on
    # the host so that no input-synthesis kernel runs on the GPU
    x, y = synth.luma_pairs_u8(N_PAIRS, H, W, seed_ref=10 + 1000 * rank, seed_dist=100000 + 1000 * rank)
    x, y = x.to(dev), y.to(dev)
    px = gbssim.plane(x)
    p = gbssim.make_params(exponents=gbssim.MSSSIM_EXPONENTS)
    wsp = gbssim.workspace(px, p, gbssim.OP_MSSSIM, dev)
    stream = torch.cuda.current_stream(dev)

    def step():
        return gbssim.msssim(x, y, ws=wsp)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize(dev)

    def timed(fn, k):
        barrier()
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(k):
            fn()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        barrier()
        ms = e0.elapsed_time(e1)
        if ws > 1:
            t = torch.tensor([ms], device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            ms = t.item()
        return ms

    # FP32 peak of this GPU, measured before the timed phase (the ALU roofline's denominator)
    fp32_peak, fp32_rates = measure_fp32_peak(gbssim, dev)
    # clocks are sampled over the whole timed phase (the main steps, the
    # scale-0 kernel, the end-to-end leg, C1 and the secondary workloads); the
    # main steps alone last only tens of milliseconds
    clk = ClockSampler(local).__enter__()
    time.sleep(0.1)  # the sampler's first line
    t_main0 = time.time()
    ms = timed(step, args.steps)
    t_main1 = time.time()
    value = ws * N_PAIRS * PX_PER_PAIR * args.steps / (ms / 1e3) / 1e6
    ms_step = ms / args.steps
    score = step()

    # Dominant kernel: the persistent MS-SSIM kernel, one launch per step over
    # all 5 levels of the 64 pairs.  Its duration is taken from the CUDA events
    # around the timed steps (the step also holds a counter memset and the
    # finaliser, under 1% of it), so the fraction is a lower bound.
    outputs = N_PAIRS * sum((h - 10) * (w - 10) for h, w in LEVELS)
    flop_step = N_PAIRS * sum((FLOP_PER_CS_OUTPUT if j < len(LEVELS) - 1 else FLOP_PER_OUTPUT) * (h - 10) * (w - 10)
                              for j, (h, w) in enumerate(LEVELS))
    achieved = flop_step / (ms_step / 1e3) / 1e12
    # secondary: the scale-0 grid kernel alone (gbssim_ssim_map on the same pairs)
    wss = gbssim.workspace(px, p, gbssim.OP_SSIM, dev)
    ms_k = timed(lambda: gbssim.ssim(x, y, ws=wss), args.steps) / args.steps
    outputs0 = N_PAIRS * (H - 10) * (W - 10)
    hbm_peak, hbm_src = _peaks()
    in_bytes = 2 * N_PAIRS * PX_PER_PAIR
    hbm_frac = in_bytes / (ms_step / 1e3) / 1e9 / hbm_peak

    # end to end: pinned host inputs through gbssim_msssim_host (host->device
    # copies of the step's pairs overlapped with the level kernels, scores
    # copied back), synchronised every step
    xh = x.cpu().pin_memory()
    yh = y.cpu().pin_memory()
    wsh = gbssim.host_workspace(xh, args.e2e_chunks)
    outh = torch.empty(N_PAIRS, dtype=torch.float64).pin_memory()
    e2e_step = lambda: gbssim.msssim_host(xh, yh, chunks=args.e2e_chunks, ws=wsh, out=outh)
    for _ in range(2):
        e2e_step()
    ke = max(2, args.steps // 5)
    ms_e2e = timed(e2e_step, ke) / ke
    e2e = {"value": ws * N_PAIRS * PX_PER_PAIR / (ms_e2e / 1e3) / 1e6, "unit": UNIT, "ms_per_step": ms_e2e,
           "chunks": args.e2e_chunks, "h2d_bytes_per_step": in_bytes, "d2h_bytes_per_step": 8 * N_PAIRS}

    c1 = c1_latency(gbssim, synth, dev)
    args.fp32_peak = fp32_peak
    extra = {}
    if not args.no_extras:
        extra = run_extras(args, gbssim, synth, x, y, dev, timed, ws)
    clk.__exit__()
    clocks = dict(clk.summary(), window="whole timed phase (main steps, scale-0 kernel, end to end, C1, "
                                         "secondary workloads), nvidia-smi every 20 ms")
    clocks_main = clk.summary(t_main0 - 0.05, t_main1 + 0.05)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": max(args.warmup, 3), "ms_per_step": ms_step, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": dict(CONFIG, parallelism="dp%d" % ws if ws > 1 else "single"),
                "gpu_launches": LAUNCHES_PER_STEP * args.steps,
                "e2e": e2e,
                "hbm_frac": hbm_frac,
                "roofline": {"bound": "alu", "kernel": "gauss11_persistent_kernel<uint8_t, UniformSource> (5 levels)",
                             "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                             "frac": achieved / fp32_peak, "traffic": _traffic(),
                             "peak_source": "measured on this GPU before the timed phase: gbssim_fp32_probe "
                                            "(independent FFMA / FFMA2 chains, 16 CTAs x 256 threads per SM, "
                                            "median of 5 launches), the larger rate",
                             "peak_probe_tflops": fp32_rates,
                             "peak_derived_tflops": FP32_PEAK_DERIVED_TFLOPS,
                             "units_per_launch": outputs, "flop_per_unit": flop_step / outputs,
                             "kernel_ms": ms_step, "hbm_peak_gbs": hbm_peak, "hbm_peak_source": hbm_src,
                             "scale0_grid_kernel": {"kernel": "gauss11_kernel<uint8_t>", "ms": ms_k,
                                                    "achieved": FLOP_PER_OUTPUT * outputs0 / (ms_k / 1e3) / 1e12,
                                                    "frac": FLOP_PER_OUTPUT * outputs0 / (ms_k / 1e3) / 1e12
                                                    / fp32_peak}},
                "c1_single_pair_256": c1,
                "clocks": clocks,
                "clocks_main_region": clocks_main,
                "score_mean": float(score.double().mean().item())}
        line.update(extra)
        if not args.no_cpu_baseline and ws == 1:
            line["cpu_baseline"] = cpu_baseline()
            if not args.no_extras:
                line["cpu_baseline"]["workloads"] = oracle_workloads()
        print(json.dumps(line))
    if ws > 1:
        dist.destroy_process_group()


def run_case(args):
    """One of the bench's workloads alone, `warmup` + `steps` calls, for
    profilers: msssim = the benchmark step itself (gbssim_msssim on the 64
    1080p pairs: one persistent launch + finaliser); scale0 = gbssim_ssim_map
    on the 64 1080p pairs (the
    scale-0 Gaussian level); box8s4 = the 8x8 stride-4 box SSIM on them;
    loss = SSIMLoss forward + backward on 32x3x512x512 fp32; ssim3d = SSIM-3D
    (11 x 11 x 5) of 40 luma frames of 1920x1080; msssim3d = MS-SSIM-3D (5
    scales) of the same frames; ragged = one MS-SSIM run of a batch plan
    over 72 ragged pairs (64 drawn from the six resolutions, 8 odd sizes;
    default tuning); pool = pooling (--pool-kind, mean by default) of the 64
    stored SSIM maps (1070 x 1910 fp32).  Prints one JSON
    line with the mean time per call (CUDA events)."""
    import torch

    from paper_2101_06354_gb300 import build

    build.build()
    from paper_2101_06354_gb300 import gbssim, synth

    dev = torch.device("cuda", 0)
    if args.case == "msssim":
        x, y = synth.luma_pairs_u8(N_PAIRS, H, W)
        x, y = x.to(dev), y.to(dev)
        wsm = gbssim.workspace(gbssim.plane(x), gbssim.make_params(exponents=gbssim.MSSSIM_EXPONENTS),
                               gbssim.OP_MSSSIM, dev)
        fn = lambda: gbssim.msssim(x, y, ws=wsm)
    elif args.case in ("scale0", "box8s4"):
        x, y = synth.luma_pairs_u8(N_PAIRS, H, W)
        x, y = x.to(dev), y.to(dev)
        kw = {} if args.case == "scale0" else dict(window="box", k=8, stride=4)
        wsc = gbssim.workspace(gbssim.plane(x), gbssim.make_params(**kw), gbssim.OP_SSIM, dev)
        fn = lambda: gbssim.ssim(x, y, ws=wsc, **kw)
    elif args.case in ("ssim3d", "msssim3d"):
        v = synth.video_yuv420_u8(40, H, W)
        vx, vy = v["y"][0].contiguous().to(dev), v["y"][1].contiguous().to(dev)
        if args.case == "ssim3d":
            fn = lambda: gbssim.ssim3d(vx, vy, kt=5, k=11)
        else:
            fn = lambda: gbssim.msssim3d(vx, vy, kt=5, k=11, scales=5)
    elif args.case == "pool":
        x, y = synth.luma_pairs_u8(N_PAIRS, H, W)
        _, qmap = gbssim.ssim(x.to(dev), y.to(dev), return_map=True)
        nq, hq, wq = qmap.shape
        pq = gbssim.Plane(qmap.data_ptr(), gbssim.F32, nq, hq, wq, qmap.stride(1), qmap.stride(0))
        wsq = gbssim.workspace(pq, gbssim.Params(), gbssim.OP_POOL, dev)
        pargs = {"mean": (), "cov": (), "minkowski": (4.0,), "fns": (), "pp": (6.0, 4000.0)}[args.pool_kind]
        fn = lambda: gbssim.ssim_pool(qmap, args.pool_kind, *pargs, ws=wsq)
    elif args.case == "ragged":
        sizes = synth.ragged_sizes(64, 8)
        xs, ys = synth.ragged_pairs_u8(sizes, device=dev)
        plan = gbssim.BatchPlan(xs, ys, multiscale=True)
        fn = plan.run
    else:
        lx, ly = synth.loss_pairs_float(32, 3, 512, 512)
        xd, yd = lx.to(dev), ly.to(dev).requires_grad_(True)
        lf = gbssim.SSIMLoss(L=1.0)

        def fn():
            yd.grad = None
            lf(xd, yd).backward()

    for _ in range(args.warmup):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    print(json.dumps({"case": args.case, "steps": args.steps, "warmup": args.warmup,
                      "ms_per_call": e0.elapsed_time(e1) / max(args.steps, 1)}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gbssim", choices=["gbssim", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the box-window and loss fwd+bwd figures")
    ap.add_argument("--e2e-chunks", type=int, default=E2E_CHUNKS,
                    help="host pipeline of the end-to-end leg: 0 streams, N >= 1 double-buffers N chunks (the "
                         "form to run under a profiler that serialises launches: a streamed launch waits for "
                         "copies on another stream)")
    ap.add_argument("--case", choices=["msssim", "scale0", "box8s4", "loss", "ssim3d", "msssim3d", "ragged", "pool"],
                    default=None,
                    help="run one secondary workload alone (for profilers) instead of the benchmark")
    ap.add_argument("--pool-kind", default="mean", choices=["mean", "cov", "minkowski", "fns", "pp"],
                    help="pooling kind of --case pool")
    args = ap.parse_args()
    if args.case:
        run_case(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gbssim(args)


if __name__ == "__main__":
    main()
