"""Pins of the oracle's error-controlled quantization (Sec. IV-A), the
unpredictable fallback, the error bound (Sec. II metric 1, Table 5) and the
adaptive interval count (Sec. IV-B)."""
import numpy as np
import pytest

from conftest import golden_path
from synthetic import fields


def _max_err(x, y):
    return float(np.max(np.abs(x.astype(np.float64) - y.astype(np.float64))))


def _range(x):
    return float(x.max()) - float(x.min())


def test_effective_eb_is_largest_float_below(szo):
    """eb_f is the largest binary32 value <= eb = eb_rel * (max - min)."""
    rng = np.random.default_rng(0)
    for _ in range(500):
        lo, hi = np.sort(rng.standard_normal(2).astype(np.float32) * 10 ** rng.uniform(-3, 3))
        rel = 10 ** rng.uniform(-7, -1)
        eb, ebf = szo.effective_eb(szo.REL, 0.0, rel, float(lo), float(hi))
        assert eb == rel * (float(hi) - float(lo))
        assert float(np.float32(ebf)) <= eb
        assert float(np.nextafter(np.float32(ebf), np.float32(np.inf))) > eb
    eb, ebf = szo.effective_eb(szo.ABS_AND_REL, 1e-3, 1e-4, 0.0, 100.0)
    assert eb == min(1e-3, 1e-4 * 100.0)


def test_truncation_bound_and_exactness(szo):
    """The truncated representation of an unpredictable value is within the
    bound (strictly), is exact for eb = 0, and keeps the sign/exponent."""
    rng = np.random.default_rng(1)
    xs = np.concatenate([rng.standard_normal(3000) * 10.0 ** rng.integers(-30, 30, 3000),
                         np.array([0.0, -0.0, 1e-40, -3e-42, 3.4e38, -1.2e-38])]).astype(np.float32)
    for eb in [0.0, 1e-45, 1e-38, 1e-8, 1e-4, 0.37, 1.0, 3e5]:
        ebf = float(np.float32(eb))
        for x in xs:
            t, tr = szo.truncate(float(x), ebf)
            assert 0 <= t <= 23
            if ebf == 0.0:
                assert np.float32(tr).view(np.uint32) == x.view(np.uint32)
            else:
                assert abs(float(x) - float(tr)) < ebf
            assert (np.float32(tr).view(np.uint32) >> 23) == (x.view(np.uint32) >> 23)


def test_quantizer_picks_nearest_interval(szo):
    """Brute force: an accepted code is the interval whose centre
    pred + q*2eb is nearest to x, the error is below eb and q stays within
    the 2^(m-1)-1 radius; a value is rejected (code 0) only when no centre
    within the radius holds it.  Binary32 rounding of x - pred and of the
    centre moves things by a few units in the last place, which the
    tolerance `slack` (in units of the interval width) allows for."""
    rng = np.random.default_rng(2)
    for _ in range(6000):
        m = int(rng.integers(2, 17))
        eb = float(np.float32(10 ** rng.uniform(-6, 0)))
        pred = float(np.float32(rng.standard_normal() * 3))
        x = float(np.float32(pred + rng.standard_normal() * eb * 10 ** rng.uniform(0, 5)))
        code, rec = szo.quantize(x, pred, eb, m)
        R = 2 ** (m - 1) - 1
        qexact = (x - pred) / (2 * eb)
        qn = int(np.floor(qexact + 0.5))
        ulp = float(np.spacing(np.float32(max(abs(x), abs(pred), abs(pred + qn * 2 * eb)))))
        slack = 2 * ulp / (2 * eb) + 4e-7 * abs(qexact) + 1e-6
        assert abs(x - rec) < eb
        if code == 0:
            assert abs(qn) > R - 1 or abs(abs(qexact - qn) - 0.5) < slack
        else:
            q = code - 2 ** (m - 1)
            assert 1 <= code <= 2 ** m - 1 and abs(q) <= R
            if abs(abs(qexact - qn) - 0.5) > slack:
                assert q == qn


def _check_bound(szo, x, **kw):
    s = szo.compress(x, **kw)
    y = szo.decompress(s)
    h = szo.header(s)
    err = _max_err(x, y)
    eb_f = h["eb_f"]
    assert err < eb_f or (eb_f == 0.0 and err == 0.0)
    return s, y, err, eb_f


@pytest.mark.parametrize("n", [1, 2])
@pytest.mark.parametrize("ebrel", [1e-2, 1e-4, 1e-6])
def test_error_bound_every_point_2d(szo, n, ebrel):
    """|x - x'| < eb at every point (Sec. II metric 1)."""
    x = fields.grf2d(64, 80, seed=5)
    _check_bound(szo, x, eb_rel=ebrel, n=n, m=0)


@pytest.mark.parametrize("n", [1, 2])
def test_error_bound_every_point_3d(szo, n):
    x = fields.blobs3d(12, 20, 24, seed=6, nblobs=6)
    for ebrel in [1e-3, 1e-5]:
        _check_bound(szo, x, eb_rel=ebrel, n=n, m=0)
    _check_bound(szo, x, mode=szo.ABS, eb_abs=1e-3, n=n, m=6)
    _check_bound(szo, x, mode=szo.ABS_AND_REL, eb_abs=1e-3, eb_rel=1e-4, n=n, m=5)


def test_max_error_reaches_bound(szo):
    """Table 5: the maximum error equals the bound to two digits (the bound
    is reached, not just respected) on a noisy field, for every eb_rel."""
    rows = [l.split() for l in open(golden_path("table5_max_error.txt"))
            if l.strip() and not l.startswith("#")]
    x = fields.grf2d(128, 128, seed=7)
    for ebrel_s, atm_s, _ in rows:
        ebrel = float(ebrel_s)
        s, y, err, eb_f = _check_bound(szo, x, eb_rel=ebrel, n=1, m=12)
        assert round(err / _range(x), 7) <= float(atm_s)
        assert float("%.1e" % (err / _range(x))) == float(atm_s) or err / eb_f > 0.95


def test_lossless_when_bound_is_zero(szo):
    """eb_abs = 0 gives an exact round trip (the lossless special case)."""
    x = fields.grf2d(40, 50, seed=8)
    s, y, err, eb_f = _check_bound(szo, x, mode=szo.ABS, eb_abs=0.0, m=8)
    assert eb_f == 0.0 and np.array_equal(x, y)


def test_constant_field(szo):
    """A constant field: one unpredictable point (the first; its prediction
    is 0) and N-1 centre codes; a zero field has no unpredictable point."""
    for c in [3.25, 0.0]:
        x = np.full((30, 40), c, np.float32)
        s, rec, codes = szo.compress(x, mode=szo.ABS, eb_abs=1e-3, m=8, want_aux=True)
        assert int((codes == 0).sum()) == (1 if c else 0)
        assert int((codes == 128).sum()) == x.size - (1 if c else 0)
        assert szo.header(s)["K"] == (1 if c else 0)
        assert np.array_equal(szo.decompress(s), x)


def test_huge_bound_single_symbol(szo):
    """With a bound larger than the data, every point takes the centre code:
    one used symbol, coded with length 1."""
    x = fields.grf2d(20, 30, seed=9)
    s, rec, codes = szo.compress(x, mode=szo.ABS, eb_abs=1e6, m=8, want_aux=True)
    h = szo.header(s)
    assert np.all(codes == 128) and h["nsym"] == 1 and h["maxlen"] == 1
    assert _max_err(x, szo.decompress(s)) < 1e6


def test_linear_field_centre_codes(szo):
    """n = 1 (n = 2 in 1D) is exact on a linear field at interior points, so
    with a dyadic bound (2 eb = 2^-9, increments multiples of it) every
    reconstruction equals the input and every interior code is the centre
    2^(m-1).  On faces the zero-padded stencil is the lower-dimensional one,
    which sees a nonzero slope: predictable, but not the centre code."""
    for shape, n in [((33,), 2), ((17, 19), 1), ((7, 9, 11), 1)]:
        x = fields.linear_field(shape)
        m = 12
        s, rec, codes = szo.compress(x, mode=szo.ABS, eb_abs=2.0 ** -10, n=n, m=m,
                                     want_aux=True)
        assert codes.ravel()[0] == 2 ** (m - 1) + 512  # first point: pred 0, x = 1.0 = 512 * 2eb
        assert np.array_equal(rec, x)
        interior = tuple(slice(n, None) for _ in shape)
        assert np.all(codes[interior] == 2 ** (m - 1))
        assert np.all(codes.ravel()[1:] != 0)


def _adaptive_1d(q_at_samples, eb=0.5):
    """1D field whose sampled differences to the previous original value are
    q*2eb exactly (dyadic), so the sampled |q| is known."""
    n = 8 * len(q_at_samples) + 1
    x = np.zeros(n, np.float64)
    v = 0.0
    for i in range(n):
        s = i // 8
        if i % 8 == 0 and s < len(q_at_samples):
            v = v + q_at_samples[s] * 2 * eb
        x[i] = v
    return x.astype(np.float32)


def test_adaptive_m_from_sampled_hit_rate(szo):
    """Sec. IV-B: the smallest m whose 2^m - 1 intervals hold a fraction
    theta of the sampled points.  |q| <= 2^(m-1)-1 needs m = 2 for |q|<=1,
    3 for |q|<=3, 4 for |q|<=7 ..."""
    # 100 samples: the first has pred 0 and diff 0 (x=... starts at q*2eb)
    qs = [0] * 1 + [1] * 60 + [3] * 30 + [7] * 9
    x = _adaptive_1d(qs)
    assert szo.choose_m(x, 1, 0.5, theta=0.60) == 2
    assert szo.choose_m(x, 1, 0.5, theta=0.61) == 2
    assert szo.choose_m(x, 1, 0.5, theta=0.62) == 3
    assert szo.choose_m(x, 1, 0.5, theta=0.91) == 3
    assert szo.choose_m(x, 1, 0.5, theta=0.92) == 4
    assert szo.choose_m(x, 1, 0.5, theta=1.0) == 4
    assert szo.choose_m(x, 1, 0.5, theta=0.0) == 2
    # nothing reaches theta -> 16
    y = _adaptive_1d([40000] * 10)
    assert szo.choose_m(y, 1, 0.5, theta=0.5) == 16


def test_adaptive_m_monotone(szo):
    """More demanding theta or a smaller bound never lowers m."""
    x = fields.grf2d(96, 96, seed=11)
    rng = _range(x)
    prev = 0
    for th in [0.5, 0.8, 0.9, 0.99, 0.999]:
        m = szo.choose_m(x, 1, np.float32(1e-4 * rng), theta=th)
        assert m >= prev
        prev = m
    prev = 0
    for e in [1e-2, 1e-3, 1e-4, 1e-5, 1e-6]:
        m = szo.choose_m(x, 1, float(np.float32(e * rng)), theta=0.99)
        assert m >= prev
        prev = m
