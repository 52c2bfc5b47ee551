"""The autotuner picks a wavefront shape and a Huffman chunk length per shape
class and persists them; the shape changes the schedule only and the chunk
length only the chunking, so after tuning every stream is byte-identical to
the oracle's stream with that chunk length (whole rows when the length is at
least the row), also after a save/load round trip, and decompresses to the
same values."""
import numpy as np
import pytest

from synthetic import fields

pytestmark = pytest.mark.gpu


def _oracle_chunk(szgb, t):
    return 0 if t["chunk"] == szgb.CHUNK_ROWS else t["chunk"]


def test_autotune_keeps_bits(szo, tmp_path):
    import torch
    from paper_1706_03791_gb300 import build
    build.build()
    from paper_1706_03791_gb300 import szgb
    cases = [(fields.blobs3d(20, 40, 44, seed=36, nblobs=8), dict(eb_rel=1e-4, m=0)),
             (fields.grf2d(301, 203, seed=32), dict(eb_rel=1e-4, m=0)),
             (fields.blobs3d(21, 45, 36, seed=39, nblobs=6), dict(eb_rel=1e-4, layers=2, m=0))]
    ctx = szgb.Context(0)
    path = str(tmp_path / "tune.txt")
    try:
        chunks = []
        for x, kw in cases:
            xd = torch.from_numpy(x).cuda()
            t = ctx.autotune(xd, reps=1, **kw)
            assert t["W"] in (1, 2, 4, 6, 8) and t["chunk"] in (szgb.CHUNK_ROWS, 128, 256, 512, 1024) and t["ms"] > 0
            chunks.append(_oracle_chunk(szgb, t))
            ref = szo.compress(x, chunk_points=chunks[-1], **kw)
            s, _ = ctx.compress(xd, **kw)
            assert np.array_equal(s.cpu().numpy(), ref)
            y = ctx.decompress(s)
            assert np.array_equal(y.cpu().numpy().view(np.uint32),
                                  szo.decompress(ref).view(np.uint32))
            # an explicit request overrides the tuned length
            s2, _ = ctx.compress(xd, chunk_points=szgb.CHUNK_ROWS, **kw)
            assert np.array_equal(s2.cpu().numpy(), szo.compress(x, **kw))
        ctx.tune_save(path)
        lines = [l for l in open(path) if not l.startswith("#")]
        assert len(lines) == len(cases)
        ctx2 = szgb.Context(0)
        ctx2.tune_load(path)
        for (x, kw), c in zip(cases, chunks):
            s, _ = ctx2.compress(torch.from_numpy(x).cuda(), **kw)
            assert np.array_equal(s.cpu().numpy(), szo.compress(x, chunk_points=c, **kw))
        bad = tmp_path / "bad.txt"
        bad.write_text("0123 99 4 1.0\n")
        with pytest.raises(szgb.SzgbError) as e:
            ctx2.tune_load(str(bad))
        assert e.value.code == szgb.ECORRUPT
        ctx2.close()
    finally:
        ctx.close()


def test_autotune_batch_keeps_bits(szo):
    import torch
    from paper_1706_03791_gb300 import build
    build.build()
    from paper_1706_03791_gb300 import szgb
    xs = [fields.grf2d(256, 256, seed=1), fields.blobs3d(12, 36, 40, seed=38, nblobs=6),
          fields.grf2d(300, 211, seed=83)]
    kw = dict(eb_rel=1e-4, m=0)
    ctx = szgb.Context(0)
    try:
        xd = [torch.from_numpy(x).cuda() for x in xs]
        t = ctx.autotune_batch(xd, kw, reps=1)
        assert t["W"] in (1, 2, 4, 6, 8) and t["chunk"] in (szgb.CHUNK_ROWS, 128, 512)
        sb, _ = ctx.compress_batch(xd, kw)
        for x, s in zip(xs, sb):
            assert np.array_equal(s.cpu().numpy(), szo.compress(x, chunk_points=_oracle_chunk(szgb, t), **kw))
        ys = ctx.decompress_batch(sb)
        for x, s, y in zip(xs, sb, ys):
            assert np.array_equal(y.cpu().numpy().view(np.uint32), szo.decompress(s.cpu().numpy()).view(np.uint32))
    finally:
        ctx.close()
