"""szgb_quality_dev (Sec. II, Metrics 1-3) against the oracle's float64
metrics: random and offset fields, unaligned views (scalar loads), an exact
reconstruction, and a reconstruction from the compressor."""
import math

import numpy as np
import pytest

from oracle.metrics import quality as oracle_quality
from synthetic import fields

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch
    from paper_1706_03791_gb300 import build
    build.build()
    from paper_1706_03791_gb300 import szgb
    assert torch.cuda.is_available()
    c = szgb.Context(0)
    yield c
    c.close()


def _check(got, ref):
    for k in ("max_abs_err", "rmse", "x_min", "x_max"):
        assert got[k] == pytest.approx(ref[k], rel=1e-10, abs=1e-300), k
    for k in ("nrmse", "max_rel_err", "psnr"):
        assert got[k] == pytest.approx(ref[k], rel=1e-9), k
    assert got["pearson"] == pytest.approx(ref["pearson"], abs=1e-10)
    assert got["n"] == ref["n"]


@pytest.mark.parametrize("n,offset,start", [(1_000_003, 0.0, 0), (4096, 1.0e4, 1), (7, -3.0, 0), (257, 0.0, 3)])
def test_random(ctx, n, offset, start):
    import torch
    rng = np.random.default_rng(n)
    x = (rng.normal(size=n + start) + offset).astype(np.float32)
    y = (x + rng.normal(scale=1e-3, size=n + start)).astype(np.float32)
    xd, yd = torch.from_numpy(x).cuda()[start:], torch.from_numpy(y).cuda()[start:]
    _check(ctx.quality(xd, yd), oracle_quality(x[start:], y[start:]))  # start > 0: unaligned, scalar loads


def test_exact(ctx):
    import torch
    x = torch.from_numpy(fields.grf2d(128, 96, seed=5)).cuda()
    q = ctx.quality(x, x.clone())
    assert q["rmse"] == 0.0 and q["max_abs_err"] == 0.0 and q["psnr"] == math.inf
    assert q["pearson"] == pytest.approx(1.0, abs=1e-12)


def test_reconstruction(ctx):
    import torch
    x = fields.blobs3d(20, 64, 48, seed=9, nblobs=6)
    xd = torch.from_numpy(x).cuda()
    s, st = ctx.compress(xd, eb_rel=1e-4, m=0)
    y = ctx.decompress(s)
    q = ctx.quality(xd, y)
    _check(q, oracle_quality(x, y.cpu().numpy()))
    assert q["max_abs_err"] < st.eb_f
