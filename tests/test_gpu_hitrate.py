"""szgb_hit_count_dev (Sec. III, Table 2) against the oracle's hit counts:
prediction from original values for 1D/2D/3D fields and n = 1..4, and from
the values the GPU compressor recorded for every layer count it carries."""
import numpy as np
import pytest

from oracle import hitrate
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


def _field(ndim):
    if ndim == 1:
        return np.cumsum(np.random.default_rng(7).normal(size=100_003)).astype(np.float32)
    if ndim == 2:
        return fields.grf2d(300, 257, seed=3, slope=5.0, noise=0.0)
    return fields.blobs3d(40, 50, 60, seed=2, turb=0.01)


@pytest.mark.parametrize("ndim", (1, 2, 3))
@pytest.mark.parametrize("n", (1, 2, 3, 4))
def test_orig_counts(ctx, ndim, n):
    import torch
    x = _field(ndim)
    xd = torch.from_numpy(x).cuda()
    span = float(x.max() - x.min())
    for eb in (0.0, 1e-4 * span, 1e-2 * span):
        assert ctx.hit_count(xd, xd, n, eb) == hitrate.hit_count(x, x, n, eb), eb


@pytest.mark.parametrize("ndim,n", [(1, 1), (1, 4), (2, 1), (2, 2), (2, 3), (3, 1), (3, 2)])
def test_decomp_counts(ctx, ndim, n):
    import torch
    x = _field(ndim)
    xd = torch.from_numpy(x).cuda()
    got = ctx.hit_rates(xd, n, eb_rel=1e-3)
    ref = hitrate.hit_rates(x, n, eb_rel=1e-3)
    assert got["eb_f"] == ref["eb_f"] and got["m"] == ref["m"]
    assert got["hits_orig"] == ref["hits_orig"]
    assert got["hits_decomp"] == ref["hits_decomp"]


def test_constant_and_bad_args(ctx):
    import torch
    from paper_1706_03791_gb300 import szgb
    x = torch.ones((6, 5, 7), dtype=torch.float32, device="cuda")
    for n in (1, 2, 3, 4):
        assert ctx.hit_count(x, x, n, 0.5) == x.numel() - n ** 3
    with pytest.raises(szgb.SzgbError):
        ctx.hit_count(x, x, 5, 0.5)
    with pytest.raises(szgb.SzgbError):
        ctx.hit_count(x, x, 1, -1.0)
