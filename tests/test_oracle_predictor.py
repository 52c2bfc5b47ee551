"""Pins of the oracle's n-layer predictor (Sec. III, Eq. predmodel, Table 1,
Theorem 1) against what the paper prints and what the mathematics fixes."""
import itertools
import math
from math import comb, factorial

import numpy as np
import pytest

from conftest import golden_path


def _table1():
    rows = {}
    for line in open(golden_path("table1_2d_predictor.txt")):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        n, k1, k2, c = map(int, line.split())
        rows.setdefault(n, {})[(k1, k2)] = c
    return rows


@pytest.mark.parametrize("n", [1, 2, 3, 4])
def test_table1_coefficients(szo, n):
    """The generic d-dimensional formula reproduces Table 1 term by term."""
    k, c = szo.terms(2, n)
    got = {(int(a[1]), int(a[2])): int(v) for a, v in zip(k, c)}
    assert all(a[0] == 0 for a in k)
    assert got == _table1()[n]


@pytest.mark.parametrize("d", [1, 2, 3, 4])
@pytest.mark.parametrize("n", [1, 2, 3, 4])
def test_term_count_and_sum(szo, d, n):
    """(n+1)^d - 1 coefficients (Algorithm 1, coefficient step); in 2D the
    n-layer subset has n(n+2) points; coefficients sum to 1, so a constant is
    predicted exactly."""
    k, c = szo.terms(d, n)
    assert len(c) == (n + 1) ** d - 1
    if d == 2:
        assert len(c) == n * (n + 2)
    assert int(c.sum()) == 1
    # every offset is in [0,n]^d, none is the point itself, all distinct
    w = k.shape[1]  # 3 columns up to 3D, 4 in 4D; absent axes are 0
    assert all(not a[:w - d].any() for a in k)
    offs = {tuple(a[w - d:]) for a in k}
    assert len(offs) == len(c)
    assert all(max(o) <= n and min(o) >= 0 and any(o) for o in offs)
    # closed form of each coefficient: -prod_j (-1)^k_j C(n, k_j)
    for a, v in zip(k, c):
        prod = 1
        for kj in a[w - d:]:
            prod *= (-1) ** int(kj) * comb(n, int(kj))
        assert v == -prod


def test_lorenzo_special_case(szo):
    """n = 1 is the Lorenzo predictor: 2D V(i,j-1)+V(i-1,j)-V(i-1,j-1);
    3D the 7-point Lorenzo stencil with signs (-1)^(|k|+1)."""
    k, c = szo.terms(3, 1)
    for a, v in zip(k, c):
        assert v == (-1) ** (int(a.sum()) + 1)


def _poly_field(shape, monomials):
    """Integer-valued polynomial sum c * prod_a x_a^e_a on the grid."""
    grids = np.meshgrid(*[np.arange(s, dtype=np.int64) for s in shape], indexing="ij")
    f = np.zeros(shape, dtype=np.int64)
    for c, ex in monomials:
        t = np.full(shape, c, dtype=np.int64)
        for g, e in zip(grids, ex):
            t = t * g ** e
        f += t
    return f


@pytest.mark.parametrize("n", [1, 2, 3])
def test_theorem_polynomial_exactness_2d(szo, n):
    """Theorem 1: with n layers the prediction equals the value of any
    polynomial surface of total degree <= 2n-1, at every point with n
    preceding layers.  Values are small integers, so every float operation
    is exact and equality is bitwise."""
    rng = np.random.default_rng(10 + n)
    side = 9
    mons = []
    for a in range(2 * n):
        for b in range(2 * n - a):
            mons.append((int(rng.integers(-3, 4)), (a, b)))
    f = _poly_field((side, side), mons)
    assert np.abs(f).max() < 2 ** 20
    V = f.astype(np.float32)
    pred = szo.predict_field(V, n)
    assert np.array_equal(pred[n:, n:], V[n:, n:])


@pytest.mark.parametrize("n", [1, 2])
def test_theorem_is_sharp(szo, n):
    """The bound is sharp: x^n y^n (degree 2n) is not reproduced; the
    residual is the mixed n-th difference, which is (n!)^2 for x^n y^n."""
    f = _poly_field((8, 8), [(1, (n, n))]).astype(np.float32)
    pred = szo.predict_field(f, n)
    res = (f - pred)[n:, n:]
    assert np.all(res == float(factorial(n) ** 2))


@pytest.mark.parametrize("d,n", [(3, 1), (3, 2), (2, 1), (2, 2), (1, 1), (1, 2)])
def test_product_structure_exactness(szo, d, n):
    """Eq. predmodel factorises: V - f = prod_a (n-th backward difference
    along a) V.  So a monomial is reproduced iff some exponent is < n; in
    particular n = 1 is exact on additive fields g(i)+h(j)(+w(k))."""
    shape = {1: (20,), 2: (9, 10), 3: (6, 7, 8)}[d]
    rng = np.random.default_rng(d * 10 + n)
    exact, inexact = [], []
    for ex in itertools.product(range(n + 2), repeat=d):
        (exact if min(ex) < n else inexact).append(ex)
    mons = [(int(rng.integers(1, 3)), e) for e in exact]
    f = _poly_field(shape, mons)
    assert np.abs(f).max() < 2 ** 22
    V = f.astype(np.float32)
    pred = szo.predict_field(V, n)
    sl = tuple(slice(n, None) for _ in range(d))
    assert np.array_equal(pred[sl], V[sl])
    # a monomial with every exponent >= n is not reproduced
    g = _poly_field(shape, [(1, tuple([n] * d))]).astype(np.float32)
    pg = szo.predict_field(g, n)
    assert not np.array_equal(pg[sl], g[sl])


@pytest.mark.parametrize("n", [1, 2])
def test_product_structure_exactness_4d(szo, n):
    """The factorisation holds in 4D (the predictor is defined for any d):
    V - f = prod over the 4 axes of the n-th backward difference, so
    monomials with an exponent below n are reproduced away from the first n
    layers and x^n y^n z^n w^n is not.  Values stay below 2^16, so every
    partial sum (at most (2^(4n) - 1) * 2^16 < 2^24) is exact."""
    shape = (4, 4, 4, 5)
    rng = np.random.default_rng(40 + n)
    cand = [e for e in itertools.product(range(n + 2), repeat=4) if min(e) < n and sum(e) <= 6]
    pick = rng.choice(len(cand), size=8, replace=False)
    mons = [(int(rng.integers(1, 3)), cand[i]) for i in pick]
    f = _poly_field(shape, mons)
    assert np.abs(f).max() < 2 ** 16
    V = f.astype(np.float32)
    pred = szo.predict_field(V, n)
    sl = tuple(slice(n, None) for _ in range(4))
    assert np.array_equal(pred[sl], V[sl])
    g = _poly_field(shape, [(1, (n, n, n, n))]).astype(np.float32)
    res = (g - szo.predict_field(g, n))[sl]
    assert np.all(res == float(factorial(n) ** 4))  # the mixed n-th difference of prod x_a^n


def test_additive_field_exact_n1(szo):
    """n = 1 predicts any g(i)+h(j) exactly away from the first row/column
    (dyadic values keep float arithmetic exact)."""
    rng = np.random.default_rng(3)
    gi = rng.integers(-100, 100, 17) / 8.0
    hj = rng.integers(-100, 100, 19) / 8.0
    V = (gi[:, None] + hj[None, :]).astype(np.float32)
    pred = szo.predict_field(V, 1)
    assert np.array_equal(pred[1:, 1:], V[1:, 1:])


def test_boundary_zero_padding(szo):
    """Neighbours outside the domain count as 0: the first point is
    predicted as 0 and the first row of a 2D field by the left neighbour."""
    V = (np.arange(12, dtype=np.float32).reshape(3, 4) + 1.0)
    pred = szo.predict_field(V, 1)
    assert pred[0, 0] == 0.0
    assert np.array_equal(pred[0, 1:], V[0, :-1])
    assert np.array_equal(pred[1:, 0], V[:-1, 0])


@pytest.mark.parametrize("n", [1, 2, 3, 4])
def test_theorem_polynomial_exactness_1d(szo, n):
    """In 1D the n-layer prediction is the extrapolation through the n
    preceding values: exact for every polynomial of degree <= n - 1 (small
    integer values, so every float operation is exact)."""
    rng = np.random.default_rng(30 + n)
    coef = rng.integers(-3, 4, size=n)
    t = np.arange(24, dtype=np.int64)
    f = sum(int(c) * t ** k for k, c in enumerate(coef))
    assert np.abs(f).max() < 2 ** 20
    V = f.astype(np.float32)
    pred = szo.predict_field(V, n)
    assert np.array_equal(pred[n:], V[n:])
    # degree n is not reproduced: the residual is the n-th difference, n! c_n
    g = (t ** n).astype(np.float32)
    res = g - szo.predict_field(g, n)
    assert np.all(res[n:] == math.factorial(n))
