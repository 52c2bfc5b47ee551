"""Huffman chunks of C points along each row on the GPU against the oracle's
chunked streams: byte-identical streams from the GPU encoder, bit-identical
reconstructions from the GPU chunk decoder, for chunk lengths from 32 points
to whole rows, ragged last chunks, 1D-4D, the hyperplane path, batches with
mixed lengths, host buffers and the no-allocation decompression."""
import numpy as np
import pytest

from synthetic import fields

pytestmark = pytest.mark.gpu


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
    ("1d-5000", lambda: fields.grf2d(1, 5000, seed=91).reshape(5000), dict(eb_rel=1e-4, m=0)),
    ("2d-97x211", lambda: fields.grf2d(97, 211, seed=92), dict(eb_rel=1e-5, m=0)),
    ("2d-n2-300x1000", lambda: fields.grf2d(300, 1000, seed=93), dict(eb_rel=1e-4, m=0, layers=2)),
    ("3d-7x19x300", lambda: fields.blobs3d(7, 19, 300, seed=94, nblobs=4), dict(eb_rel=1e-5, m=0)),
    ("3d-n2-12x40x77", lambda: fields.blobs3d(12, 40, 77, seed=95, nblobs=4), dict(eb_rel=1e-4, m=0, layers=2)),
]
CHUNKS = [32, 64, 128, 256, 512, 1024, 4096]


@pytest.mark.parametrize("name,gen,kw", CASES, ids=[c[0] for c in CASES])
def test_chunked_streams_match_oracle(env, szo, name, gen, kw):
    torch, szgb, ctx = env
    x = np.ascontiguousarray(gen())
    xd = torch.from_numpy(x).cuda()
    _, rec, _ = szo.compress(x, want_aux=True, **kw)
    for C in CHUNKS:
        ref = szo.compress(x, chunk_points=C, **kw)
        s, st = ctx.compress(xd, chunk_points=C, **kw)
        assert np.array_equal(s.cpu().numpy(), ref), C
        assert st.stream_bytes == ref.size
        info = szgb.stream_info(s.cpu().numpy())
        assert info["chunk_points"] == (C if C < x.shape[-1] else szgb.CHUNK_ROWS)
        y = ctx.decompress(s)  # the device path (one-field graph)
        assert np.array_equal(_bits(y.cpu().numpy()), _bits(rec)), C
        yo = ctx.decompress(torch.from_numpy(ref).cuda())  # the oracle's stream
        assert np.array_equal(_bits(yo.cpu().numpy()), _bits(rec)), C


def test_chunked_direct_and_host_paths(env, szo):
    torch, szgb, ctx = env
    x = fields.blobs3d(9, 33, 130, seed=96, nblobs=4)
    kw = dict(eb_rel=1e-4, m=0, chunk_points=64)
    ref, rec, _ = szo.compress(x, want_aux=True, **kw)
    ctx.set_graphs(False)  # the direct path
    try:
        s, _ = ctx.compress(torch.from_numpy(x).cuda(), **kw)
        assert np.array_equal(s.cpu().numpy(), ref)
        y = ctx.decompress(s)
        assert np.array_equal(_bits(y.cpu().numpy()), _bits(rec))
    finally:
        ctx.set_graphs(True)
    sh, _ = ctx.compress(x, **kw)  # host buffers
    assert np.array_equal(sh, ref)
    yh = ctx.decompress(sh)
    assert np.array_equal(_bits(yh), _bits(rec))
    s2, r2, c2, _ = ctx.compress_trace(torch.from_numpy(x).cuda(), **kw)
    assert np.array_equal(s2.cpu().numpy(), ref) and np.array_equal(_bits(r2.cpu().numpy()), _bits(rec))


def test_chunked_hyperplane_and_4d(env, szo):
    torch, szgb, ctx = env
    x3 = fields.blobs3d(6, 20, 90, seed=97, nblobs=3)
    kw3 = dict(eb_rel=1e-4, m=0, layers=3, chunk_points=32)
    ref3, rec3, _ = szo.compress(x3, want_aux=True, **kw3)
    s3, _ = ctx.compress(torch.from_numpy(x3).cuda(), **kw3)
    assert np.array_equal(s3.cpu().numpy(), ref3)
    assert np.array_equal(_bits(ctx.decompress(s3).cpu().numpy()), _bits(rec3))
    x4 = fields.blobs3d(6, 8, 70, seed=98, nblobs=3).reshape(2, 3, 8, 70)
    kw4 = dict(eb_rel=1e-4, m=8, chunk_points=32)
    ref4, rec4, _ = szo.compress(x4, want_aux=True, **kw4)
    s4, _ = ctx.compress(torch.from_numpy(np.ascontiguousarray(x4)).cuda(), **kw4)
    assert np.array_equal(s4.cpu().numpy(), ref4)
    assert np.array_equal(_bits(ctx.decompress(s4).cpu().numpy()), _bits(rec4))


def test_chunked_batch_mixed(env, szo):
    torch, szgb, ctx = env
    xs = [fields.grf2d(120, 300, seed=99), fields.blobs3d(10, 30, 200, seed=100, nblobs=4),
          fields.grf2d(1, 3000, seed=101).reshape(3000), fields.grf2d(64, 64, seed=102)]
    kws = [dict(eb_rel=1e-4, m=0, chunk_points=32), dict(eb_rel=1e-4, m=0, chunk_points=128),
           dict(eb_rel=1e-3, m=0, chunk_points=1024), dict(eb_rel=1e-4, m=0, chunk_points=szgb.CHUNK_ROWS)]
    refs = [szo.compress(x, want_aux=True, **{k: v for k, v in kw.items() if k != "chunk_points"},
                         chunk_points=(0 if kw["chunk_points"] == szgb.CHUNK_ROWS else kw["chunk_points"]))
            for x, kw in zip(xs, kws)]
    xd = [torch.from_numpy(x).cuda() for x in xs]
    for rep in range(2):  # captured, then replayed
        sb, _ = ctx.compress_batch(xd, kws)
        for i, (s, (sref, rec, _)) in enumerate(zip(sb, refs)):
            assert np.array_equal(s.cpu().numpy(), sref), i
        ys = ctx.decompress_batch(sb)
        for i, (y, (_, rec, _)) in enumerate(zip(ys, refs)):
            assert np.array_equal(_bits(y.cpu().numpy()), _bits(rec)), i


def test_chunked_noalloc(env, szo):
    torch, szgb, ctx = env
    x = fields.blobs3d(8, 40, 257, seed=103, nblobs=4)
    ref, rec, _ = szo.compress(x, want_aux=True, eb_rel=1e-4, m=0, chunk_points=64)
    s = torch.from_numpy(ref).cuda()
    out = torch.full(x.shape, float("nan"), dtype=torch.float32, device="cuda")
    rc = szgb.decompress_noalloc(s, out, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert rc == szgb.OK, szgb.strerror(rc)
    assert np.array_equal(_bits(out.cpu().numpy()), _bits(rec))


def test_invalid_chunk_rejected(env):
    torch, szgb, ctx = env
    xd = torch.from_numpy(fields.grf2d(16, 100, seed=104)).cuda()
    for C in (16, 48, 100):
        with pytest.raises(szgb.SzgbError) as e:
            ctx.compress(xd, eb_rel=1e-3, m=8, chunk_points=C)
        assert e.value.code == szgb.EINVAL


# chunk counts around the chunk-offset scan's tile of 2048 entries and its
# 1024-tile limit for the two-kernel form: one tile (partial and full), two
# tiles, and 1028 tiles (the three-kernel form)
SCAN_CASES = [
    ("1-tile-partial", lambda: fields.grf2d(40, 100, seed=101), dict(chunk_points=32), 160),
    ("1-tile-full", lambda: fields.grf2d(64, 1024, seed=102), dict(chunk_points=32), 2048),
    ("2-tiles", lambda: fields.grf2d(2049, 32, seed=103), dict(), 2049),
    ("1028-tiles", lambda: fields.walk3d(1028, 2048, 8, seed=104), dict(), 1028 * 2048),
]


@pytest.mark.parametrize("name,gen,ckw,nchunks", SCAN_CASES, ids=[c[0] for c in SCAN_CASES])
def test_chunk_offset_scan_sizes(env, szo, name, gen, ckw, nchunks):
    torch, szgb, ctx = env
    x = np.ascontiguousarray(gen())
    kw = dict(eb_rel=1e-4, m=0, **ckw)
    ref, rec, _ = szo.compress(x, want_aux=True, **kw)
    rows = int(np.prod(x.shape[:-1]))
    C = ckw.get("chunk_points", 0)
    per_row = -(-x.shape[-1] // C) if 0 < C < x.shape[-1] else 1
    assert rows * per_row == nchunks
    s, st = ctx.compress(torch.from_numpy(x).cuda(), **kw)
    assert np.array_equal(s.cpu().numpy(), ref)
    y = ctx.decompress(s)
    assert np.array_equal(_bits(y.cpu().numpy()), _bits(rec))
