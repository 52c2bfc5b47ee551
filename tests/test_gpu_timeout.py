"""The wavefront's bounded device-side waits, run out on purpose without
faulting or hanging the GPU: a test hook leaves one work item unrun, so its
consumers poll halo words that are never written.  With a short wait limit
every call must return SZGB_ETIMEOUT promptly (every CTA gave up, published
an aborted state and exited), and the same context must then give the
oracle's stream and reconstruction again."""
import time

import numpy as np
import pytest

from synthetic import fields

pytestmark = pytest.mark.gpu

LIMIT_NS = 20_000_000  # 20 ms


@pytest.fixture(scope="module")
def env():
    import torch
    from paper_1706_03791_gb300 import build
    build.build()
    from paper_1706_03791_gb300 import szgb
    c = szgb.Context(0)
    yield torch, szgb, c
    c.close()


def _bits(a):
    return np.ascontiguousarray(a).reshape(-1).view(np.uint32)


CASES = [
    # 3D: 5 plane blocks x 4 row blocks; item 0 feeds every other item
    ("3d-item0", lambda: fields.blobs3d(40, 100, 60, seed=81, nblobs=6), dict(eb_rel=1e-4, m=0), 0),
    # 3D: an item in the middle of the pipeline (plane block 1, row block 2)
    ("3d-item6", lambda: fields.blobs3d(40, 100, 60, seed=81, nblobs=6), dict(eb_rel=1e-4, m=0), 6),
    # 2D, two layers: row blocks of 256 rows, item 1 of 4
    ("2d-n2-item1", lambda: fields.grf2d(1000, 300, seed=82), dict(eb_rel=1e-4, m=0, layers=2), 1),
]


@pytest.mark.parametrize("name,gen,kw,item", CASES, ids=[c[0] for c in CASES])
def test_wait_runs_out_then_context_recovers(env, szo, name, gen, kw, item):
    torch, szgb, ctx = env
    x = np.ascontiguousarray(gen())
    sref, rec, _ = szo.compress(x, want_aux=True, **kw)
    xd = torch.from_numpy(x).cuda()
    good = torch.from_numpy(sref).cuda()
    ctx.debug_set_wait_limit(LIMIT_NS)
    try:
        ctx.debug_skip_item(item)
        for op in ("compress", "decompress"):
            t0 = time.perf_counter()
            with pytest.raises(szgb.SzgbError) as e:
                if op == "compress":
                    ctx.compress(xd, **kw)
                else:
                    ctx.decompress(good)
            dt = time.perf_counter() - t0
            assert e.value.code == szgb.ETIMEOUT, (op, e.value.code)
            # far below the default 4 s limit: the short limit applied
            assert dt < 2.0, (op, dt)
        # a batch of two fields: the item is skipped in both
        with pytest.raises(szgb.SzgbError) as e:
            ctx.compress_batch([xd, xd], kw)
        assert e.value.code == szgb.ETIMEOUT
    finally:
        ctx.debug_skip_item(-1)
        ctx.debug_set_wait_limit(0)
    # the same context, hook off: the oracle's bytes and values again
    for _ in range(2):
        s, st = ctx.compress(xd, **kw)
        assert np.array_equal(s.cpu().numpy(), sref)
        y = ctx.decompress(s)
        assert np.array_equal(_bits(y.cpu().numpy()), _bits(rec))
    sb, _ = ctx.compress_batch([xd, xd], kw)
    for si in sb:
        assert np.array_equal(si.cpu().numpy(), sref)


def test_hook_arguments(env):
    torch, szgb, ctx = env
    with pytest.raises(szgb.SzgbError):
        ctx.debug_skip_item(-2)
