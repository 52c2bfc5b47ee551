"""Whole-path pins of the oracle: bit-exact round trip of the recorded
(decompressed) values, independence of the traversal order (any order that
respects the dependency DAG gives the same bytes), header consistency and
error handling."""
import numpy as np
import pytest

from synthetic import fields


CASES = [
    ("1d", lambda: fields.grf2d(1, 700, seed=20).reshape(700), dict(eb_rel=1e-4, m=0)),
    ("2d", lambda: fields.grf2d(37, 53, seed=21), dict(eb_rel=1e-4, m=8)),
    ("2d-n2", lambda: fields.grf2d(31, 45, seed=22), dict(eb_rel=1e-3, n=2, m=0)),
    ("3d", lambda: fields.blobs3d(9, 13, 17, seed=23, nblobs=4), dict(eb_rel=1e-4, m=0)),
    ("3d-n2", lambda: fields.blobs3d(8, 10, 12, seed=24, nblobs=4), dict(eb_rel=1e-5, n=2, m=0)),
    ("3d-m16", lambda: fields.blobs3d(7, 9, 11, seed=25, nblobs=4), dict(eb_rel=1e-6, m=16)),
]


@pytest.mark.parametrize("name,gen,kw", CASES, ids=[c[0] for c in CASES])
def test_round_trip_bit_exact(szo, name, gen, kw):
    x = gen()
    s, rec, codes = szo.compress(x, want_aux=True, **kw)
    y = szo.decompress(s)
    assert y.shape == x.shape
    assert np.array_equal(y.view(np.uint32), rec.view(np.uint32))
    h = szo.header(s)
    assert h["total_bytes"] == s.size and h["K"] == int((codes == 0).sum())
    assert codes.max() < (1 << h["m"])
    assert h["nchunks"] == x.size // x.shape[-1]


@pytest.mark.parametrize("name,gen,kw", CASES, ids=[c[0] for c in CASES])
def test_hyperplane_order_same_bytes(szo, name, gen, kw):
    """The prediction uses only neighbours with smaller i+j+k, so a
    hyperplane (wavefront) traversal gives the identical stream."""
    x = gen()
    a = szo.compress(x, order=0, **kw)
    b = szo.compress(x, order=1, **kw)
    assert np.array_equal(a, b)


def test_nonfinite_rejected(szo):
    x = fields.grf2d(8, 8, seed=1)
    for bad in [np.nan, np.inf, -np.inf]:
        y = x.copy()
        y[3, 4] = bad
        assert szo.compress_rc(y, eb_rel=1e-3, m=8) == szo.ENONFINITE


def test_invalid_arguments(szo):
    x = fields.grf2d(8, 8, seed=1)
    assert szo.compress_rc(x, eb_rel=1e-3, m=1) == szo.EINVAL
    assert szo.compress_rc(x, eb_rel=1e-3, m=17) == szo.EINVAL
    assert szo.compress_rc(x, eb_rel=-1.0, m=8) == szo.EINVAL
    assert szo.compress_rc(x, eb_rel=1e-3, n=0, m=8) == szo.EINVAL


def test_corrupt_streams_rejected(szo):
    x = fields.grf2d(20, 24, seed=2)
    s = szo.compress(x, eb_rel=1e-3, m=8)
    assert szo.decompress_rc(s[:100]) in (szo.EINVAL, szo.ECORRUPT)
    bad = s.copy()
    bad[0] ^= 0xFF
    assert szo.decompress_rc(bad) == szo.ECORRUPT
    assert szo.decompress_rc(s[:-5]) == szo.ECORRUPT
    bad = s.copy()
    bad[10] = 40  # m out of range
    assert szo.decompress_rc(bad) == szo.ECORRUPT


def test_compression_factor_on_smooth_field(szo):
    """Smooth 3D field at eb_rel 1e-4 compresses well (CF >> 1), the bit
    rate matches CF (BR * CF = 32, Sec. II metric 4)."""
    x = fields.blobs3d(20, 40, 48, seed=26, nblobs=8)
    s = szo.compress(x, eb_rel=1e-4, m=0)
    cf = x.nbytes / s.size
    br = s.size * 8 / x.size
    assert cf > 3.0 and abs(br * cf - 32.0) < 1e-9
