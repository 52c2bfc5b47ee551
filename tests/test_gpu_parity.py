"""GPU path vs the CPU oracle: byte-identical streams, bit-identical recorded
(decompressed) values and quantization codes, and bit-identical
decompression, through the C ABI, on seeded synthetic fields of the paper's
shapes at sizes that span several tiles, warps and CTAs with ragged tails."""
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


def _check(ctx, szo, x, **kw):
    import torch
    xd = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    s_gpu, rec, codes, st = ctx.compress_trace(xd, **kw)
    s_ref, rec_ref, codes_ref = szo.compress(x, want_aux=True, **kw)
    sg = s_gpu.cpu().numpy()
    rg = rec.cpu().numpy()
    cg = codes.cpu().numpy().view(np.uint16)
    assert np.array_equal(cg, codes_ref), "codes differ at %s" % (np.argwhere(cg != codes_ref)[:5],)
    assert np.array_equal(_bits(rg), _bits(rec_ref)), "recorded values differ"
    assert sg.size == s_ref.size, "stream length %d vs %d" % (sg.size, s_ref.size)
    diff = np.nonzero(sg != s_ref)[0]
    assert diff.size == 0, "stream bytes differ from offset %d" % diff[0]
    y = ctx.decompress(s_gpu)
    assert np.array_equal(_bits(y.cpu().numpy()), _bits(rec_ref)), "GPU decompression differs"
    y2 = ctx.decompress(s_ref)  # oracle stream through the host path
    assert np.array_equal(_bits(y2), _bits(rec_ref))
    eb = szo.header(s_ref)["eb_f"]
    err = np.abs(rec_ref.astype(np.float64) - x)
    assert (err < eb).all() or eb == 0.0
    return st


CASES = [
    ("1d", lambda: fields.grf2d(1, 777, seed=31).reshape(777), dict(eb_rel=1e-4, m=8)),
    ("2d-256", lambda: fields.grf2d(256, 256, seed=1), dict(eb_rel=1e-4, layers=1, m=8)),
    ("2d-ragged", lambda: fields.grf2d(301, 203, seed=32), dict(eb_rel=1e-4, m=0)),
    ("2d-multicta", lambda: fields.grf2d(700, 130, seed=33), dict(eb_rel=1e-3, m=0)),
    ("2d-n2", lambda: fields.grf2d(97, 140, seed=34), dict(eb_rel=1e-4, layers=2, m=0)),
    ("2d-n2-ragged", lambda: fields.grf2d(290, 61, seed=35), dict(eb_rel=1e-3, layers=2, m=10)),
    ("3d", lambda: fields.blobs3d(20, 40, 44, seed=36, nblobs=8), dict(eb_rel=1e-4, m=0)),
    ("3d-ragged", lambda: fields.blobs3d(19, 70, 37, seed=37, nblobs=8), dict(eb_rel=1e-4, m=0)),
    ("3d-eb6", lambda: fields.blobs3d(12, 36, 40, seed=38, nblobs=6), dict(eb_rel=1e-6, m=0)),
    ("3d-n2", lambda: fields.blobs3d(21, 45, 36, seed=39, nblobs=6), dict(eb_rel=1e-4, layers=2, m=0)),
    ("3d-n2-eb6", lambda: fields.blobs3d(10, 34, 29, seed=40, nblobs=6), dict(eb_rel=1e-6, layers=2, m=0)),
    ("3d-abs", lambda: fields.blobs3d(9, 33, 20, seed=41, nblobs=4), dict(mode=0, eb_abs=1e-3, m=6)),
    ("3d-both", lambda: fields.blobs3d(9, 33, 20, seed=42, nblobs=4), dict(mode=2, eb_abs=1e-3, eb_rel=1e-5, m=12)),
    ("2d-m16", lambda: fields.grf2d(80, 90, seed=43), dict(eb_rel=1e-7, m=16)),
    ("2d-m2", lambda: fields.grf2d(50, 64, seed=44), dict(eb_rel=1e-2, m=2)),
    # n = 3, 4 (1D and 2D)
    ("1d-n3", lambda: fields.grf2d(1, 777, seed=47).reshape(777), dict(eb_rel=1e-4, layers=3, m=0)),
    ("1d-n4", lambda: fields.grf2d(1, 1030, seed=48).reshape(1030), dict(eb_rel=1e-3, layers=4, m=8)),
    ("2d-n3", lambda: fields.grf2d(97, 140, seed=49), dict(eb_rel=1e-4, layers=3, m=0)),
    ("2d-n3-multicta", lambda: fields.grf2d(700, 130, seed=50), dict(eb_rel=1e-3, layers=3, m=0)),
    ("2d-n4-ragged", lambda: fields.grf2d(290, 61, seed=51), dict(eb_rel=1e-4, layers=4, m=10)),
]


@pytest.mark.parametrize("name,gen,kw", CASES, ids=[c[0] for c in CASES])
def test_parity(ctx, szo, name, gen, kw):
    _check(ctx, szo, gen(), **kw)


def test_lossless_and_constant(ctx, szo):
    x = fields.grf2d(40, 52, seed=45)
    _check(ctx, szo, x, mode=0, eb_abs=0.0, m=8)
    _check(ctx, szo, np.full((33, 70), 2.5, np.float32), mode=0, eb_abs=1e-3, m=8)
    _check(ctx, szo, np.zeros((5, 6, 7), np.float32), eb_rel=1e-4, m=0)
    _check(ctx, szo, fields.linear_field((9, 40, 44)), mode=0, eb_abs=2.0 ** -10, m=12)


def test_tiny_shapes(ctx, szo):
    for shape in [(1,), (2,), (5,), (1, 1), (1, 9), (9, 1), (3, 5), (1, 1, 1), (2, 1, 3), (1, 33, 5), (40, 1, 1)]:
        rng = np.random.default_rng(len(shape) * 100 + sum(shape))
        x = rng.standard_normal(shape).astype(np.float32)
        _check(ctx, szo, x, eb_rel=1e-2, m=0)


def test_negative_zero_and_subnormals(ctx, szo):
    rng = np.random.default_rng(7)
    x = rng.standard_normal((37, 45)).astype(np.float32) * 1e-3
    x[::5, ::3] = -0.0
    x[1::7, ::2] = 0.0
    x[2::9, 1::4] = np.float32(3e-40)
    _check(ctx, szo, x, mode=0, eb_abs=1e-4, m=8)
    _check(ctx, szo, x, mode=0, eb_abs=0.0, m=8)


def test_full_size_3d(ctx, szo):
    """The 100x500x500 workload the benchmark times, in its launch
    configuration: whole stream and reconstruction against the oracle."""
    x = fields.workload_3d()
    for kw in [dict(eb_rel=1e-4, m=0), dict(eb_rel=1e-4, layers=2, m=0)]:
        _check(ctx, szo, x, **kw)


def test_errors(ctx, szo):
    import torch
    from paper_1706_03791_gb300 import szgb
    x = fields.grf2d(30, 40, seed=46)
    y = x.copy()
    y[3, 7] = np.nan
    with pytest.raises(szgb.SzgbError) as e:
        ctx.compress(torch.from_numpy(y).cuda(), eb_rel=1e-3, m=8)
    assert e.value.code == szgb.ENONFINITE
    y[3, 7] = np.inf
    with pytest.raises(szgb.SzgbError) as e:
        ctx.compress(y, eb_rel=1e-3, m=8)
    assert e.value.code == szgb.ENONFINITE
    s = szo.compress(x, eb_rel=1e-3, m=8)
    bad = s.copy()
    bad[128] = 200  # codebook symbol out of order
    bad[129] = 255
    with pytest.raises(szgb.SzgbError) as e:
        ctx.decompress(bad)
    assert e.value.code == szgb.ECORRUPT
    with pytest.raises(szgb.SzgbError) as e:
        ctx.decompress(s[:-3])
    assert e.value.code == szgb.ECORRUPT
    small = np.empty(10, np.uint8)
    with pytest.raises(szgb.SzgbError) as e:
        ctx.compress(x, out=small, eb_rel=1e-3, m=8)
    assert e.value.code == szgb.ETRUNC
    x3 = torch.from_numpy(fields.blobs3d(6, 20, 24, seed=52, nblobs=3)).cuda()
    with pytest.raises(szgb.SzgbError) as e:  # a bad parameter refuses the whole batch before any launch
        ctx.compress_batch([x3, x3], [dict(eb_rel=1e-3, m=8, layers=3), dict(eb_rel=1e-3, m=1)])
    assert e.value.code == szgb.EINVAL
    # the context stays usable after errors
    _check(ctx, szo, x, eb_rel=1e-3, m=8)


# large alphabets: white noise at a small absolute bound spreads the codes
# over a 16-bit alphabet (> 8192 used symbols: radix-sorted leaves; > 16384:
# leaf weights in global memory)
WIDE = [((300, 300), 1e-4, 91), ((400, 400), 4e-5, 92)]


@pytest.mark.parametrize("shape,eb,seed", WIDE, ids=["wide-radix", "wide-global"])
def test_parity_large_alphabet(ctx, szo, shape, eb, seed):
    x = np.random.default_rng(seed).random(shape).astype(np.float32)
    st = _check(ctx, szo, x, mode=0, eb_abs=eb, m=16)
    assert st.nsym > 8192
