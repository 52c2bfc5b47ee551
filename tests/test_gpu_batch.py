"""Batched compression and decompression (one persistent wavefront launch for
many fields, captured in a CUDA graph) against the CPU oracle: every field's
stream is byte-identical to the oracle's stream of that field alone, and every
reconstruction bit-identical -- the result of a field is the same alone and in
the mix.  Fields of mixed dimension, size, layer count and bound."""
import numpy as np
import pytest

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


def _bits(a):
    return np.ascontiguousarray(a).view(np.uint32)


MIX = [
    (lambda: fields.grf2d(64, 72, seed=61), dict(eb_rel=1e-4, m=8)),
    (lambda: fields.grf2d(301, 203, seed=62), dict(eb_rel=1e-4, m=0)),
    (lambda: fields.blobs3d(19, 70, 37, seed=63, nblobs=8), dict(eb_rel=1e-4, m=0)),
    (lambda: fields.grf2d(1, 900, seed=64).reshape(900), dict(eb_rel=1e-3, m=8)),
    (lambda: fields.blobs3d(5, 33, 44, seed=65, nblobs=4), dict(mode=0, eb_abs=1e-3, m=6)),
    (lambda: fields.grf2d(97, 140, seed=66), dict(eb_rel=1e-4, layers=2, m=0)),
    (lambda: fields.blobs3d(21, 45, 36, seed=67, nblobs=6), dict(eb_rel=1e-5, layers=2, m=0)),
    (lambda: fields.grf2d(700, 130, seed=68), dict(eb_rel=1e-3, m=0)),
    (lambda: fields.grf2d(120, 90, seed=69), dict(eb_rel=1e-4, layers=3, m=0)),
    (lambda: fields.grf2d(1, 500, seed=71).reshape(500), dict(eb_rel=1e-3, layers=4, m=8)),
]


def _run(ctx, szo, graphs, reps):
    import torch
    xs = [np.ascontiguousarray(g()) for g, _ in MIX]
    kws = [kw for _, kw in MIX]
    xd = [torch.from_numpy(x).cuda() for x in xs]
    refs = [szo.compress(x, want_aux=True, **kw) for x, kw in zip(xs, kws)]
    ctx.set_graphs(graphs)
    for _ in range(reps):  # the second call replays the captured graph
        streams, stats = ctx.compress_batch(xd, kws)
        for i, (s, (sref, rec, _)) in enumerate(zip(streams, refs)):
            sg = s.cpu().numpy()
            assert sg.size == sref.size, "field %d: stream length %d vs %d" % (i, sg.size, sref.size)
            assert np.array_equal(sg, sref), "field %d: stream bytes differ" % i
            assert stats[i].stream_bytes == sref.size
        ys = ctx.decompress_batch(streams)
        for i, (y, (_, rec, _)) in enumerate(zip(ys, refs)):
            assert np.array_equal(_bits(y.cpu().numpy()), _bits(rec)), "field %d: reconstruction differs" % i
    ctx.set_graphs(True)


def test_batch_graph(ctx, szo):
    _run(ctx, szo, graphs=True, reps=2)


def test_batch_direct(ctx, szo):
    _run(ctx, szo, graphs=False, reps=1)


def test_batch_matches_single(ctx):
    import torch
    x = [torch.from_numpy(fields.grf2d(256, 256, seed=1)).cuda(),
         torch.from_numpy(fields.blobs3d(12, 36, 40, seed=38, nblobs=6)).cuda()]
    kw = dict(eb_rel=1e-4, m=0)
    sb, _ = ctx.compress_batch(x, kw)
    for xi, si in zip(x, sb):
        s1, _ = ctx.compress(xi, **kw)
        assert torch.equal(s1.cpu(), si.cpu())


def test_batch_error_reporting(ctx):
    import torch
    from paper_1706_03791_gb300 import szgb
    good = torch.from_numpy(fields.grf2d(40, 50, seed=70)).cuda()
    bad = good.clone()
    bad[3, 7] = float("nan")
    with pytest.raises(szgb.SzgbError) as e:
        ctx.compress_batch([good, bad], dict(eb_rel=1e-4, m=8))
    assert e.value.code == szgb.ENONFINITE
    # the context stays usable
    s, _ = ctx.compress_batch([good], dict(eb_rel=1e-4, m=8))
    assert s[0].numel() > 128


def test_single_field_both_paths(ctx, szo):
    """A single device field runs the direct path (graphs off) or the one-field
    batched path replayed from a graph (graphs on, the default): both give the
    oracle's stream and reconstruction, on the first call and on replays."""
    import torch
    cases = [MIX[1], MIX[2], MIX[3], MIX[5]]
    try:
        for graphs in (False, True):
            ctx.set_graphs(graphs)
            for g, kw in cases:
                x = np.ascontiguousarray(g())
                sref, rec, _ = szo.compress(x, want_aux=True, **kw)
                xd = torch.from_numpy(x).cuda()
                for _ in range(2):
                    s, st = ctx.compress(xd, **kw)
                    assert np.array_equal(s.cpu().numpy(), sref)
                    assert st.stream_bytes == sref.size
                    y = ctx.decompress(s)
                    assert np.array_equal(_bits(y.cpu().numpy()), _bits(rec))
    finally:
        ctx.set_graphs(True)


def test_capped_wavefront_grid(ctx, szo):
    """A cap on the persistent wavefront's CTAs (szgb_set_wave_ctas) changes
    the schedule only: with 1, 7 and 40 CTAs, graphs on and off, the batch's
    streams and reconstructions are the oracle's."""
    import torch
    from paper_1706_03791_gb300 import szgb
    xs = [np.ascontiguousarray(g()) for g, _ in MIX]
    kws = [kw for _, kw in MIX]
    refs = [szo.compress(x, want_aux=True, **kw) for x, kw in zip(xs, kws)]
    xd = [torch.from_numpy(x).cuda() for x in xs]
    try:
        for cap in (1, 7, 40):
            ctx.set_wave_ctas(cap)
            for graphs in (True, False):
                ctx.set_graphs(graphs)
                ss, _ = ctx.compress_batch(xd, kws)
                for i, (s, (sref, rec, _)) in enumerate(zip(ss, refs)):
                    assert np.array_equal(s.cpu().numpy(), sref), (cap, graphs, i)
                ys = ctx.decompress_batch(ss)
                for i, (y, (_, rec, _)) in enumerate(zip(ys, refs)):
                    assert np.array_equal(_bits(y.cpu().numpy()), _bits(rec)), (cap, graphs, i)
        with pytest.raises(szgb.SzgbError):
            ctx.set_wave_ctas(-1)
    finally:
        ctx.set_wave_ctas(0)
        ctx.set_graphs(True)
