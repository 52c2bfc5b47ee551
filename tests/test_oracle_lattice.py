"""Pins of the oracle's lattice variant (a separately labelled, fully
parallel form; not the paper's method): every point within the bound; the
integer residuals are the mixed differences of the lattice field, checked by
array shifts and inverted by cumulative sums (numpy, not the oracle's
recurrence); lattice-aligned linear fields give zero interior residuals;
outliers are stored exactly."""
import numpy as np
import pytest

from synthetic import fields


def _lattice_ref(x, eb_f):
    """(p, ok) from the definition, in binary32: p = rint(x * inv) with
    inv = 1 / (2 eb_f); ok when |x - v| < eb_f or x == v for v = p * 2 eb_f."""
    eb = np.float32(eb_f)
    twoeb = np.float32(2.0) * eb
    inv = np.float32(1.0) / twoeb
    p = np.rint(x.astype(np.float32) * inv).astype(np.int64)
    v = p.astype(np.float32) * twoeb
    ok = (np.abs(x - v) < eb) | (x == v)
    return p, v, ok


def _mixed_diff(p, n=1):
    """r = prod over axes of (1 - shift)^n applied to p, zero outside."""
    r = p.copy()
    for ax in range(p.ndim):
        for _ in range(n):
            sh = np.zeros_like(r)
            sl = [slice(None)] * p.ndim
            sl2 = [slice(None)] * p.ndim
            sl[ax] = slice(1, None)
            sl2[ax] = slice(0, -1)
            sh[tuple(sl)] = r[tuple(sl2)]
            r = r - sh
    return r


CASES = [
    (lambda: fields.grf2d(70, 90, seed=101), dict(eb_rel=1e-4, m=0), 1),
    (lambda: fields.grf2d(33, 47, seed=102), dict(eb_rel=1e-3, m=8, n=2), 2),
    (lambda: fields.blobs3d(9, 20, 31, seed=103, nblobs=4), dict(eb_rel=1e-4, m=0), 1),
    (lambda: fields.blobs3d(7, 13, 17, seed=104, nblobs=3), dict(mode=0, eb_abs=1e-3, m=6), 1),
    (lambda: fields.grf2d(1, 500, seed=105).reshape(500), dict(eb_rel=1e-4, m=0), 1),
]


@pytest.mark.parametrize("gen,kw,n", CASES)
def test_lattice_bound_residuals_inverse(szo, gen, kw, n):
    x = gen()
    s, rec, codes = szo.compress_lattice(x, want_aux=True, **kw)
    h = szo.header(s)
    assert h["lattice"] == 1
    eb_f = h["eb_f"]
    y = szo.decompress(s)
    # the bound, at every point
    assert np.all(np.abs(y.astype(np.float64) - x) < eb_f)
    assert np.array_equal(y.view(np.uint32), rec.view(np.uint32))
    p, v, ok = _lattice_ref(x, eb_f)
    # reconstruction: the lattice value where it is within the bound, else x
    assert np.array_equal(y.view(np.uint32), np.where(ok, v, x).view(np.uint32))
    # residuals by array shifts; codes are residuals + center where small
    r = _mixed_diff(p, n)
    center = 1 << (h["m"] - 1)
    small = ok & (np.abs(r) <= center - 1)
    assert np.array_equal(codes[small].astype(np.int64), r[small] + center)
    assert np.all(codes[~small] == 0) and h["K"] == int((~small).sum())
    # the inverse: n cumulative sums per axis give p back
    q = r.copy()
    for ax in range(x.ndim):
        for _ in range(n):
            q = np.cumsum(q, axis=ax)
    assert np.array_equal(q, p)


def test_lattice_linear_field_interior_zero(szo):
    # a field on the lattice: x = (3 i - 2 j + 5) * 2 eb, eb = 2^-10 (exact)
    eb = 2.0 ** -10
    i, j = np.meshgrid(np.arange(40), np.arange(50), indexing="ij")
    x = ((3 * i - 2 * j + 5) * (2 * eb)).astype(np.float32)
    s, rec, codes = szo.compress_lattice(x, mode=0, eb_abs=eb, m=8, want_aux=True)
    assert np.array_equal(rec, x)  # every value is a lattice value
    center = 128
    assert np.all(codes[1:, 1:] == center)  # interior residuals are 0
    assert codes[0, 0] == center + 5         # first point: no neighbours


def test_lattice_outliers_exact(szo):
    # values far apart force residuals beyond the radius: stored exactly
    x = np.random.default_rng(106).random((20, 30)).astype(np.float32) * 1000.0
    s, rec, codes = szo.compress_lattice(x, mode=0, eb_abs=1e-3, m=4, want_aux=True)
    y = szo.decompress(s)
    assert np.all(np.abs(y.astype(np.float64) - x) < 1e-3)
    assert np.count_nonzero(codes == 0) > x.size // 2


def test_lattice_rejects(szo):
    x = fields.grf2d(16, 16, seed=107)
    with pytest.raises(RuntimeError):
        szo.compress_lattice(x * 1e6, mode=0, eb_abs=1e-6, m=8)    # lattice integers >= 2^30
    assert szo.compress_rc(x, mode=0, eb_abs=0.0, m=8) == 0        # exact path: lossless allowed
    with pytest.raises(RuntimeError):
        szo.compress_lattice(x, mode=0, eb_abs=0.0, m=8)            # lattice: needs eb > 0
    x2 = x.copy()
    x2[3, 3] = np.nan
    with pytest.raises(RuntimeError):
        szo.compress_lattice(x2, eb_rel=1e-4)
