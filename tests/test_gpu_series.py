"""GPU parity of temporal pooling of frame-score series (gbssim_series_pool,
Section "Spatio-temporal Aggregation of Quality Scores") against
oracle/pooling.py.  Both sides work in fp64: order statistics must match
exactly, sums to 1e-12 relative (summation order differs)."""
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


def _series():
    r = np.random.default_rng(21)
    return {
        "frames120": r.uniform(0.55, 0.99, (3, 120)),
        "ties": np.round(r.uniform(0.5, 1.0, (2, 257)) * 20) / 20,
        "one": np.array([[0.8125]]),
        "max": r.uniform(0.3, 1.0, (1, 4096)),
    }


KINDS = [("mean", (), P.mean), ("cov", (), P.cov), ("gm", (), P.gm), ("hm", (), P.hm),
         ("minkowski", (4.0,), lambda v: P.mink(v, 4.0)), ("dw", (0.5,), lambda v: P.dw(v, 0.5)),
         ("md", (2.0, 2.0), lambda v: P.md(v, 2.0, 2.0)), ("gm_dssim", (), P.gm_dssim),
         ("hm_dssim", (), P.hm_dssim), ("pp", (10.0, 4.0), lambda v: P.pp(v, 10.0, 4.0)),
         ("w_am", (1,), lambda v: P.windowed(v, 1, "am")), ("w_am", (50,), lambda v: P.windowed(v, min(50, v.size), "am")),
         ("w_gm", (80,), lambda v: P.windowed(v, min(80, v.size), "gm")),
         ("w_hm", (7,), lambda v: P.windowed(v, min(7, v.size), "hm")),
         ("w_cov", (5,), lambda v: P.windowed(v, min(5, v.size), "cov"))]
EXACT = [("median", (), P.median), ("percentile", (10.0,), lambda v: P.percentile(v, 10.0)), ("fns", (), P.fns),
         ("percentile", (100.0,), lambda v: P.percentile(v, 100.0))]


@pytest.mark.parametrize("name", ["frames120", "ties", "one", "max"])
@pytest.mark.parametrize("kind,args,f", EXACT)
def test_series_order_statistics_exact(g, name, kind, args, f):
    s = _series()[name]
    got = g.series_pool(torch.tensor(s, device=DEV), kind, *args).cpu().tolist()
    assert got == [f(row) for row in s]


@pytest.mark.parametrize("name", ["frames120", "ties", "one", "max"])
@pytest.mark.parametrize("kind,args,f", KINDS)
def test_series_kinds(g, name, kind, args, f):
    s = _series()[name]
    if kind.startswith("w_"):
        args = (min(args[0], s.shape[1]),)
    got = g.series_pool(torch.tensor(s, device=DEV), kind, *args).cpu().tolist()
    for a, b in zip(got, [f(row) for row in s]):
        if math.isnan(b):
            assert math.isnan(a)
        else:
            assert abs(a - b) <= 1e-12 * max(1.0, abs(b)), (kind, a, b)


def test_series_strided_rows(g):
    s = np.random.default_rng(3).uniform(0.4, 1.0, (4, 100))
    t = torch.zeros((4, 128), dtype=torch.float64, device=DEV)
    t[:, :100] = torch.tensor(s)
    got = g.series_pool(t[:, :100], "fns").cpu().tolist()
    assert got == [P.fns(row) for row in s]


def test_series_rejects_bad_arguments(g):
    s = torch.rand((1, 10), dtype=torch.float64, device=DEV)
    with pytest.raises(g.GbssimError):
        g.series_pool(s, "w_am", 11)          # window longer than the series
    with pytest.raises(g.GbssimError):
        g.series_pool(s, "w_gm", 2.5)         # non-integer window
    with pytest.raises(g.GbssimError):
        g.series_pool(torch.rand((1, 4097), dtype=torch.float64, device=DEV), "mean")
