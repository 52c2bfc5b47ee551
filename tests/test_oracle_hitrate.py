"""The oracle's prediction hitting rate (Sec. III, Table 2) pinned to closed
forms, a brute-force count on a tiny field, the inclusive boundary, and its
relation to the quantizer's centre code (Sec. IV-A)."""
import itertools

import numpy as np
import pytest

from oracle import szo
from oracle.hitrate import hit_count, hit_rates
from synthetic import fields


@pytest.mark.parametrize("ndim,n", list(itertools.product((1, 2, 3), (1, 2, 3, 4))))
def test_constant_orig_closed_form(ndim, n):
    # On a constant c the n-layer prediction with zero padding is
    # c * (1 - prod_a A(i_a)), A(i) = sum_{k <= min(i, n)} (-1)^k C(n, k): A(i) = 0
    # for i >= n and (-1)^i C(n-1, i) otherwise, so exactly the n^d points with
    # every index below n miss (by at least |c|) and the others hit.
    shape = {1: (23,), 2: (9, 7), 3: (6, 5, 7)}[ndim]
    for c in (1.0, -0.75):
        x = np.full(shape, c, np.float32)
        assert hit_count(x, x, n, 0.5 * abs(c)) == x.size - n ** ndim


@pytest.mark.parametrize("ndim", (1, 2, 3))
@pytest.mark.parametrize("m", (2, 16))
def test_constant_decomp_one_layer(ndim, m):
    # 1 layer on a constant field: the origin is predicted as 0 (a miss); it is
    # recorded within eb of c, and every later 1-layer prediction is a signed
    # sum of that one recorded value that collapses to it exactly, so every
    # other point hits and keeps it.
    shape = {1: (40,), 2: (8, 11), 3: (5, 6, 7)}[ndim]
    x = np.full(shape, 1.0, np.float32)
    r = hit_rates(x, 1, mode=szo.ABS, eb_abs=1e-3, m=m)
    assert r["hits_orig"] == x.size - 1
    assert r["hits_decomp"] == x.size - 1


def test_inclusive_bound():
    # "not larger than the error bound": a difference equal to eb is a hit
    x = np.array([0.0, 0.5, 0.5], np.float32)  # 1 layer: predictions 0, 0, 0.5
    assert hit_count(x, x, 1, 0.5) == 3
    assert hit_count(x, x, 1, np.nextafter(0.5, 0.0)) == 2


def _brute_1layer_2d(x, v, eb):
    # Lorenzo 1-layer predictor written out: left + up - upper-left, values
    # outside the field 0; float64 arithmetic
    n0, n1 = x.shape
    hits = 0
    for i in range(n0):
        for j in range(n1):
            a = float(v[i, j - 1]) if j > 0 else 0.0
            b = float(v[i - 1, j]) if i > 0 else 0.0
            c = float(v[i - 1, j - 1]) if i > 0 and j > 0 else 0.0
            hits += abs(float(x[i, j]) - (a + b - c)) <= eb
    return hits


def test_brute_force_tiny():
    rng = np.random.default_rng(11)
    x = np.cumsum(np.cumsum(rng.normal(size=(7, 9)), 0), 1).astype(np.float32)
    v = (x + rng.uniform(-0.05, 0.05, size=x.shape)).astype(np.float32)
    for vv in (x, v):
        f = szo.predict_field(vv, 1).astype(np.float64)
        d = np.sort(np.abs(x.astype(np.float64) - f).ravel())
        for k in (5, 20, 40):  # bounds halfway between two differences: no rounding ties
            eb = 0.5 * (d[k] + d[k + 1])
            assert hit_count(x, vv, 1, eb) == _brute_1layer_2d(x, vv, eb) == k + 1


@pytest.mark.parametrize("n", (1, 2, 3, 4))
def test_centre_code_implies_hit(n):
    # the centre code needs |x - f| < eb_f, so it counts a subset of the hits
    x = fields.grf2d(96, 80, seed=5, slope=5.0, noise=0.0)
    r = hit_rates(x, n, eb_rel=1e-3)
    centre = int(np.count_nonzero(r["codes"] == (1 << (r["m"] - 1))))
    assert centre <= r["hits_decomp"] <= centre + 2
    assert r["hits_decomp"] > 0


def test_table2_shape_on_smooth_field():
    # On a smooth field the 2-layer predictor wins on original values while
    # the 1-layer one wins on decompressed values (the comparison of Table 2)
    x = fields.grf2d(192, 192, seed=3, slope=6.0, noise=0.0)
    r1, r2 = hit_rates(x, 1, eb_rel=1e-4), hit_rates(x, 2, eb_rel=1e-4)
    assert r2["R_orig"] > r1["R_orig"]
    assert r1["R_decomp"] > r2["R_decomp"]


def test_interval_hit_rate_and_suggestion():
    # a field whose prediction errors need more than m = 2's single pair of
    # side intervals: the rate falls with smaller m and the suggestion asks
    # for one more bit exactly when the rate is below theta
    from oracle.hitrate import interval_hit_rate, suggest_m
    x = fields.grf2d(64, 64, seed=8)
    rates = {}
    for m in (2, 4, 8, 12):
        _, _, codes = szo.compress(x, eb_rel=1e-4, m=m, want_aux=True)
        r = interval_hit_rate(codes)
        assert r == 1.0 - np.count_nonzero(codes == 0) / codes.size
        rates[m] = r
        assert suggest_m(codes, m, 0.99) == (min(m + 1, 16) if r < 0.99 else m)
    assert rates[2] < rates[4] < rates[8] <= rates[12]
    assert suggest_m(np.zeros(10, np.uint16), 16, 0.5) == 16  # no m above 16
    assert suggest_m(np.ones(10, np.uint16), 3, 1.0) == 3      # every point in an interval
