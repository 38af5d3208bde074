"""GPU parity of the pooling family on stored maps (gbssim_ssim_pool, Section
"Spatio-temporal Aggregation of Quality Scores") against oracle/pooling.py
applied to the same float32 maps.  Order statistics (percentile, median,
five-number summary) are selected exactly and must match the oracle's sorted
values bit for bit; moment kinds sum fp32 terms, so they are compared at
1e-6 relative (the pooled-value tolerance)."""
import math

import numpy as np
import pytest
import torch

from oracle import pooling as P

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
def maps(g):
    from paper_2101_06354_gb300 import synth

    x, y = synth.luma_pairs_u8(3, 200, 232)
    _, q = g.ssim(x.to(DEV), y.to(DEV), return_map=True)
    r = np.random.default_rng(11)
    extra = {
        "ssim": q,
        "signed": torch.tensor(r.uniform(-0.6, 1.0, (2, 97, 131)), dtype=torch.float32, device=DEV),
        "ties": torch.tensor(np.round(r.uniform(0.2, 1.0, (2, 64, 70)) * 16) / 16, dtype=torch.float32, device=DEV),
        "single": torch.tensor([[[0.75]]], dtype=torch.float32, device=DEV),
        "ones": torch.ones((1, 9, 13), dtype=torch.float32, device=DEV),
    }
    return extra


ORDER = [("median", (), P.median), ("percentile", (10.0,), lambda v: P.percentile(v, 10.0)),
         ("percentile", (0.0,), lambda v: P.percentile(v, 0.0)), ("percentile", (100.0,), lambda v: P.percentile(v, 100.0)),
         ("percentile", (6.5,), lambda v: P.percentile(v, 6.5)), ("fns", (), P.fns)]
MOMENT = [("mean", (), P.mean), ("cov", (), P.cov), ("minkowski", (4.0,), lambda v: P.mink(v, 4.0)),
          ("minkowski", (0.125,), lambda v: P.mink(v, 0.125)), ("dw", (1.0,), lambda v: P.dw(v, 1.0)),
          ("dw", (0.25,), lambda v: P.dw(v, 0.25)), ("md", (2.0, 1.0), lambda v: P.md(v, 2.0, 1.0)),
          ("md", (1.0, 3.0), lambda v: P.md(v, 1.0, 3.0)), ("gm_dssim", (), P.gm_dssim),
          ("hm_dssim", (), P.hm_dssim), ("pp", (6.0, 4000.0), lambda v: P.pp(v, 6.0, 4000.0)),
          ("pp", (25.0, 4.0), lambda v: P.pp(v, 25.0, 4.0))]


def _refs(m, f):
    a = m.double().cpu().numpy()
    return [f(a[i]) for i in range(a.shape[0])]


@pytest.mark.parametrize("name", ["ssim", "signed", "ties", "single"])
@pytest.mark.parametrize("kind,args,f", ORDER)
def test_order_statistics_exact(g, maps, name, kind, args, f):
    m = maps[name]
    got = g.ssim_pool(m, kind, *args).cpu().tolist()
    assert got == _refs(m, f)


@pytest.mark.parametrize("name", ["ssim", "signed", "ties", "single"])
@pytest.mark.parametrize("kind,args,f", MOMENT)
def test_moment_kinds(g, maps, name, kind, args, f):
    m = maps[name]
    got = g.ssim_pool(m, kind, *args).cpu().tolist()
    for a, b in zip(got, _refs(m, f)):
        if math.isnan(b):
            assert math.isnan(a)
        else:
            assert abs(a - b) <= 1e-6 * max(1.0, abs(b)), (kind, args, a, b)


@pytest.mark.parametrize("kind,args,f", ORDER + [("percentile", (80.0,), lambda v: P.percentile(v, 80.0))])
def test_order_statistics_crowded_and_spread(g, kind, args, f):
    """Selection first bins the values over [min, max] and selects among the
    wanted bins' values when they hold at most 65536 of them together, else
    it runs the radix passes.  Image 0: 80% of 102400 values equal one
    number (its bin overflows the candidate buffer: the radix passes); image
    1: the same values spread (the value-bin path); image 2: a narrow cluster
    near 1 and a long tail, as SSIM maps have; images 3 and 4: values over
    [-5, 5] and over [0, 255], maps that are not SSIM maps."""
    r = np.random.default_rng(5)
    n = 320 * 320
    crowd = r.uniform(0.2, 1.0, n)
    crowd[r.permutation(n)[: int(0.8 * n)]] = 0.875
    spread = r.uniform(-0.3, 1.0, n)
    tail = np.where(r.uniform(size=n) < 0.9, 1.0 - r.exponential(0.004, n), r.uniform(0.0, 1.0, n))
    wide = r.uniform(-5.0, 5.0, n)
    pixels = r.uniform(0.0, 255.0, n)
    m = torch.tensor(np.stack([crowd, spread, tail, wide, pixels]).reshape(5, 320, 320), dtype=torch.float32,
                     device=DEV)
    got = g.ssim_pool(m, kind, *args).cpu().tolist()
    assert got == _refs(m, f)


def test_degenerate_all_ones(g, maps):
    m = maps["ones"]
    assert g.ssim_pool(m, "gm_dssim").item() == 0.0
    assert g.ssim_pool(m, "hm_dssim").item() == 0.0
    assert g.ssim_pool(m, "minkowski", 2.0).item() == 0.0
    assert math.isnan(g.ssim_pool(m, "dw", 1.0).item())
    assert g.ssim_pool(m, "cov").item() == 0.0
    assert g.ssim_pool(m, "fns").item() == 1.0


def test_pitched_maps_and_full_size(g):
    from paper_2101_06354_gb300 import synth

    x, y = synth.luma_pairs_u8(2, 1080, 1920)
    _, q = g.ssim(x.to(DEV), y.to(DEV), return_map=True)
    big = torch.zeros((2, q.shape[1], q.shape[2] + 7), dtype=torch.float32, device=DEV)
    big[:, :, :q.shape[2]] = q
    view = big[:, :, :q.shape[2]]  # row pitch 1917 floats
    for kind, args, f in (("fns", (), P.fns), ("percentile", (10.0,), lambda v: P.percentile(v, 10.0))):
        assert g.ssim_pool(view, kind, *args).cpu().tolist() == _refs(q, f)
    got = g.ssim_pool(view, "cov").cpu().tolist()
    for a, b in zip(got, _refs(q, P.cov)):
        assert abs(a - b) <= 1e-6 * max(1.0, abs(b))


@pytest.mark.parametrize("kw", [dict(), dict(window="box", k=8, stride=4), dict(window="gaussian", k=7, sigma=1.0)])
def test_local_mean_matches_oracle(g, kw):
    import oracle
    from paper_2101_06354_gb300 import synth

    x, _ = synth.luma_pairs_u8(2, 90, 117)
    got = g.local_mean(x.to(DEV), **kw).cpu().double().numpy()
    k, s = kw.get("k", 11), kw.get("stride", 1)
    w = oracle.window(kw.get("window", "gaussian"), k, kw.get("sigma", 1.5))
    for i in range(2):
        ref = P.local_mean(x[i].numpy(), w, s)
        assert np.abs(got[i] - ref).max() <= 1e-6 * 255


@pytest.mark.parametrize("a,b", [(0.0, 0.0), (40.0, 30.0), (100.0, 50.0), (60.0, 0.0)])
def test_luminance_weighted_pooling(g, maps, a, b):
    from paper_2101_06354_gb300 import synth

    x, y = synth.luma_pairs_u8(3, 200, 232)
    _, q = g.ssim(x.to(DEV), y.to(DEV), return_map=True)
    mu = g.local_mean(x.to(DEV))
    got = g.ssim_pool_lw(q, mu, a, b).cpu().tolist()
    qn, mn = q.double().cpu().numpy(), mu.double().cpu().numpy()
    for i in range(3):
        ref = P.lw(qn[i], mn[i], a, b)
        assert abs(got[i] - ref) <= 1e-6, (a, b, got[i], ref)
    base = g.ssim_pool(q, "mean").cpu().tolist()
    if a == 0.0 and b == 0.0:
        assert all(abs(u - v) <= 1e-7 for u, v in zip(got, base))
