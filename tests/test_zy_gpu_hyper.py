"""The GPU's hyperplane kernels against the oracle: 3D fields with n = 3 and 4
layers, and 4D fields with n = 1..4 (Sec. III, Eq. predmodel in four
dimensions).  Byte-identical streams, bit-identical recorded values, codes
and reconstructions, on fields that span many hyperplanes with ragged
extents, plus unit extents, an absolute bound, a tight bound, fixed and
adaptive m and host buffers; the same fields inside batches beside
wavefront fields.  This file runs after the other GPU tests."""
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


CASES = [
    ("n3", lambda: fields.blobs3d(13, 37, 29, seed=61, nblobs=6), dict(eb_rel=1e-4, layers=3, m=0)),
    ("n4", lambda: fields.blobs3d(11, 23, 41, seed=62, nblobs=6), dict(eb_rel=1e-3, layers=4, m=0)),
    ("n3-abs-m8", lambda: fields.blobs3d(9, 17, 33, seed=63, nblobs=4), dict(mode=0, eb_abs=1e-3, layers=3, m=8)),
    ("n4-eb6", lambda: fields.blobs3d(7, 19, 21, seed=64, nblobs=4), dict(eb_rel=1e-6, layers=4, m=0)),
    ("n3-unit-extents", lambda: fields.blobs3d(1, 1, 70, seed=65, nblobs=2), dict(eb_rel=1e-4, layers=3, m=0)),
    ("n4-thin", lambda: fields.blobs3d(2, 45, 3, seed=66, nblobs=3), dict(eb_rel=1e-4, layers=4, m=10)),
]


@pytest.mark.parametrize("name,gen,kw", CASES, ids=[c[0] for c in CASES])
def test_parity(ctx, name, gen, kw):
    import torch
    from oracle import szo
    x = gen()
    xd = torch.from_numpy(x).cuda()
    s_gpu, rec, codes, st = ctx.compress_trace(xd, **kw)
    s_ref, rec_ref, codes_ref = szo.compress(x, want_aux=True, **kw)
    assert np.array_equal(codes.cpu().numpy().view(np.uint16), codes_ref), "codes differ"
    assert np.array_equal(rec.cpu().numpy().view(np.uint32), rec_ref.view(np.uint32)), "recorded values differ"
    assert np.array_equal(s_gpu.cpu().numpy(), s_ref), "stream bytes differ"
    y = ctx.decompress(s_gpu)
    assert np.array_equal(y.cpu().numpy().view(np.uint32), rec_ref.view(np.uint32)), "reconstruction differs"
    err = np.abs(x.astype(np.float64) - y.cpu().numpy().astype(np.float64))
    assert np.all((err < st.eb_f) | (x == y.cpu().numpy()))


def test_plain_calls_and_host_buffers(ctx):
    # the plain (non-trace) compression and the host-buffer paths give the same bytes
    import torch
    from oracle import szo
    x = fields.blobs3d(8, 21, 26, seed=67, nblobs=4)
    kw = dict(eb_rel=1e-4, layers=3, m=0)
    ref = szo.compress(x, **kw)
    s_dev, _ = ctx.compress(torch.from_numpy(x).cuda(), **kw)
    assert np.array_equal(s_dev.cpu().numpy(), ref)
    s_host, _ = ctx.compress(x, **kw)
    assert np.array_equal(np.asarray(s_host), ref)
    y = ctx.decompress(np.asarray(ref))
    assert np.array_equal(y.view(np.uint32), szo.decompress(ref).view(np.uint32))


def test_batches_carry_hyperplane_fields(ctx):
    """A batch mixing wavefront fields with 3D n = 3, 4 and 4D fields: the
    latter run on the hyperplane kernels after the batch's wavefront, and
    every stream and reconstruction equals the oracle's."""
    import torch
    from oracle import szo
    xs = [fields.blobs3d(6, 20, 24, seed=68, nblobs=3), fields.blobs3d(7, 18, 21, seed=69, nblobs=3),
          _field4((3, 4, 9, 13), seed=70), fields.grf2d(45, 61, seed=71), fields.blobs3d(5, 9, 30, seed=72, nblobs=3),
          _field4((2, 3, 5, 40), seed=73)]
    kws = [dict(eb_rel=1e-3, layers=4, m=0), dict(eb_rel=1e-4, layers=1, m=0), dict(eb_rel=1e-4, layers=2, m=0),
           dict(eb_rel=1e-4, layers=2, m=0), dict(eb_rel=1e-4, layers=3, m=9), dict(eb_rel=1e-3, layers=1, m=0)]
    refs = [szo.compress(x, **kw) for x, kw in zip(xs, kws)]
    for graphs in (True, False):
        ctx.set_graphs(graphs)
        ss, sts = ctx.compress_batch([torch.from_numpy(x).cuda() for x in xs], kws)
        for i, (s, ref) in enumerate(zip(ss, refs)):
            assert np.array_equal(s.cpu().numpy(), ref), i
            assert sts[i].status == 0 and sts[i].stream_bytes == ref.size
        ys = ctx.decompress_batch([torch.from_numpy(np.ascontiguousarray(r)).cuda() for r in refs])
        for i, (y, ref) in enumerate(zip(ys, refs)):
            assert tuple(y.shape) == xs[i].shape
            assert np.array_equal(y.cpu().numpy().view(np.uint32), szo.decompress(ref).view(np.uint32)), i
    ctx.set_graphs(True)


def test_4d_from_host_memory(ctx):
    """szgb_compress with ndim = 4 takes a host array as any other field."""
    from oracle import szo
    x = _field4((3, 5, 8, 11), seed=74)
    kw = dict(eb_rel=1e-4, layers=2, m=0)
    s, st = ctx.compress(x, **kw)
    assert np.array_equal(np.asarray(s), szo.compress(x, **kw))
    y = ctx.decompress(np.asarray(s))
    assert y.shape == x.shape
    assert np.array_equal(y.view(np.uint32), szo.decompress(np.asarray(s)).view(np.uint32))


def _field4(shape, seed):
    rng = np.random.default_rng(seed)
    g = np.meshgrid(*[np.linspace(0, 1, n) for n in shape], indexing="ij")
    f = np.sin(3 * g[0] + 2 * g[1]) * np.cos(2 * g[2] - g[3]) + 0.5 * g[3] ** 2
    f += rng.normal(scale=1e-3, size=shape)
    return f.astype(np.float32)


CASES4 = [
    ("4d-n1", (5, 6, 7, 9), dict(eb_rel=1e-3, layers=1, m=0)),
    ("4d-n2", (4, 7, 6, 11), dict(eb_rel=1e-4, layers=2, m=0)),
    ("4d-n3-m8", (6, 5, 5, 8), dict(eb_rel=1e-3, layers=3, m=8)),
    ("4d-n4-abs", (5, 5, 6, 6), dict(mode=0, eb_abs=1e-3, layers=4, m=0)),
    ("4d-unit", (1, 1, 3, 40), dict(eb_rel=1e-4, layers=2, m=0)),
    ("4d-samples", (9, 10, 9, 17), dict(eb_rel=1e-4, layers=1, m=0)),  # several adaptive-m samples per axis
]


@pytest.mark.parametrize("name,shape,kw", CASES4, ids=[c[0] for c in CASES4])
def test_parity_4d(ctx, name, shape, kw):
    import torch
    from oracle import szo
    x = _field4(shape, seed=sum(shape))
    xd = torch.from_numpy(x).cuda()
    s_gpu, rec, codes, st = ctx.compress_trace(xd, **kw)
    s_ref, rec_ref, codes_ref = szo.compress(x, want_aux=True, **kw)
    assert np.array_equal(codes.cpu().numpy().view(np.uint16), codes_ref), "codes differ"
    assert np.array_equal(rec.cpu().numpy().view(np.uint32), rec_ref.view(np.uint32)), "recorded values differ"
    assert np.array_equal(s_gpu.cpu().numpy(), s_ref), "stream bytes differ"
    y = ctx.decompress(s_gpu)
    assert tuple(y.shape) == shape
    assert np.array_equal(y.cpu().numpy().view(np.uint32), rec_ref.view(np.uint32)), "reconstruction differs"
    y2 = ctx.decompress(np.asarray(s_ref))  # the oracle's stream through the host path
    assert np.array_equal(y2.view(np.uint32), rec_ref.view(np.uint32))
    s_plain, _ = ctx.compress(xd, **kw)
    assert np.array_equal(s_plain.cpu().numpy(), s_ref)


@pytest.mark.parametrize("n", [1, 2, 3, 4])
def test_hit_counts_4d(ctx, n):
    # szgb_hit_count_dev on 4D fields against the oracle's count (Sec. III)
    import torch
    from oracle import hitrate
    x = _field4((5, 6, 7, 9), seed=70 + n)
    xd = torch.from_numpy(x).cuda()
    span = float(x.max() - x.min())
    for eb in (0.0, 1e-3 * span, 1e-2 * span):
        assert ctx.hit_count(xd, xd, n, eb) == hitrate.hit_count(x, x, n, eb), eb
    r = ctx.hit_rates(xd, n, eb_rel=1e-3)
    ref = hitrate.hit_rates(x, n, eb_rel=1e-3)
    assert r["hits_orig"] == ref["hits_orig"] and r["hits_decomp"] == ref["hits_decomp"]
