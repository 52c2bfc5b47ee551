"""The lattice variant on the GPU (separately labelled; not the paper's
method) against the oracle's lattice variant: byte-identical streams,
bit-identical reconstructions and codes, every point within the bound."""
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
    c = szgb.Context(0)
    yield c
    c.close()


CASES = [
    ("2d", lambda: fields.grf2d(256, 256, seed=1), dict(eb_rel=1e-4, m=0)),
    ("2d-ragged-n2", lambda: fields.grf2d(301, 203, seed=111), dict(eb_rel=1e-3, layers=2, m=0)),
    ("3d", lambda: fields.blobs3d(19, 70, 37, seed=112, nblobs=8), dict(eb_rel=1e-4, m=0)),
    ("3d-n2", lambda: fields.blobs3d(12, 36, 40, seed=113, nblobs=6), dict(eb_rel=1e-5, layers=2, m=0)),
    ("1d", lambda: fields.grf2d(1, 5000, seed=114).reshape(5000), dict(eb_rel=1e-4, m=8)),
    ("outliers", lambda: (np.random.default_rng(115).random((64, 70)) * 1000).astype(np.float32),
     dict(mode=0, eb_abs=1e-3, m=4)),
]


@pytest.mark.parametrize("name,gen,kw", CASES, ids=[c[0] for c in CASES])
def test_lattice_parity(ctx, szo, name, gen, kw):
    import torch
    x = np.ascontiguousarray(gen())
    s_ref, rec_ref, codes_ref = szo.compress_lattice(x, want_aux=True, **kw)
    xd = torch.from_numpy(x).cuda()
    s_gpu, rec, codes, st = ctx.compress_trace(xd, variant=1, **kw)
    sg = s_gpu.cpu().numpy()
    assert np.array_equal(codes.cpu().numpy().view(np.uint16), codes_ref)
    assert np.array_equal(rec.cpu().numpy().view(np.uint32), rec_ref.view(np.uint32))
    assert sg.size == s_ref.size and np.array_equal(sg, s_ref)
    y = ctx.decompress(s_gpu)
    assert np.array_equal(y.cpu().numpy().view(np.uint32), rec_ref.view(np.uint32))
    eb = szo.header(s_ref)["eb_f"]
    assert np.all(np.abs(rec_ref.astype(np.float64) - x) < eb)
    # the plain call gives the same stream; the host path decodes the oracle's
    s2, _ = ctx.compress(xd, variant=1, **kw)
    assert np.array_equal(s2.cpu().numpy(), s_ref)
    assert np.array_equal(ctx.decompress(s_ref).view(np.uint32), rec_ref.view(np.uint32))


def test_lattice_rejections(ctx):
    import torch
    from paper_1706_03791_gb300 import szgb
    x = torch.from_numpy(fields.grf2d(40, 40, seed=116)).cuda()
    with pytest.raises(szgb.SzgbError) as e:
        ctx.compress(x, variant=1, mode=0, eb_abs=0.0, m=8)     # no lattice at eb = 0
    assert e.value.code == szgb.EINVAL
    with pytest.raises(szgb.SzgbError) as e:
        ctx.compress(x * 1e6, variant=1, mode=0, eb_abs=1e-6, m=8)  # integers >= 2^30
    assert e.value.code == szgb.EINVAL
    with pytest.raises(szgb.SzgbError) as e:  # n <= 2 only
        ctx.compress(x, variant=1, eb_rel=1e-4, layers=3)
    assert e.value.code == szgb.EUNSUPPORTED


def test_lattice_in_batches(ctx):
    """A lattice-variant field in a batch runs on its own kernels: the same
    bytes as the single-field call, beside a field on the wavefront."""
    import torch
    x = torch.from_numpy(fields.grf2d(40, 40, seed=116)).cuda()
    y = torch.from_numpy(fields.grf2d(33, 70, seed=117)).cuda()
    ss, _ = ctx.compress_batch([x, y], [dict(eb_rel=1e-4, variant=1), dict(eb_rel=1e-4)])
    s1, _ = ctx.compress(x, eb_rel=1e-4, variant=1)
    s2, _ = ctx.compress(y, eb_rel=1e-4)
    assert torch.equal(ss[0], s1) and torch.equal(ss[1], s2)
    ys = ctx.decompress_batch(ss)
    assert torch.equal(ys[0].view(torch.int32), ctx.decompress(s1).view(torch.int32))
    assert torch.equal(ys[1].view(torch.int32), ctx.decompress(s2).view(torch.int32))
