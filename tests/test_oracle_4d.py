"""The oracle's 4D form of the method (Sec. III: the predictor is defined for
any number of dimensions; Sec. IV: quantization and coding do not depend on
it).  Pinned by the error bound, the round trip, the hyperplane-order
invariance, the reduction to the 3D stream when the slowest extent is 1, and
the constant-field closed form of the hitting rate."""
import numpy as np
import pytest

from oracle import hitrate, szo


def _field4(shape, seed):
    # smooth separable-plus-mixed 4D field with a little noise
    rng = np.random.default_rng(seed)
    g = np.meshgrid(*[np.linspace(0, 1, s) for s in shape], indexing="ij")
    f = np.sin(3 * g[0] + 2 * g[1]) * np.cos(2 * g[2] - g[3]) + 0.5 * g[3] ** 2
    f += rng.normal(scale=1e-3, size=shape)
    return f.astype(np.float32)


@pytest.mark.parametrize("n", [1, 2, 3, 4])
@pytest.mark.parametrize("m", [0, 3, 8])
def test_bound_and_round_trip(n, m):
    x = _field4((5, 6, 7, 9), seed=n * 10 + m)
    s, rec, codes = szo.compress(x, eb_rel=1e-3, n=n, m=m, want_aux=True)
    hdr = szo.header(s)
    assert hdr["ndim"] == 4 and hdr["dims"] == x.shape
    eb_f = hdr["eb_f"]
    err = np.abs(x.astype(np.float64) - rec.astype(np.float64))
    assert np.all((err < eb_f) | (x == rec))
    y = szo.decompress(s)
    assert y.shape == x.shape
    assert np.array_equal(y.view(np.uint32), rec.view(np.uint32))
    assert int(np.count_nonzero(codes == 0)) == hdr["K"]


def test_abs_bound_and_unpredictables():
    x = _field4((4, 5, 6, 7), seed=1)
    x[2, 3, 1, 4] = 50.0  # an outlier no interval of m = 4 holds
    s, rec, codes = szo.compress(x, mode=szo.ABS, eb_abs=1e-3, n=1, m=4, want_aux=True)
    assert codes[2, 3, 1, 4] == 0
    assert np.all(np.abs(x.astype(np.float64) - rec) < np.float32(1e-3))
    assert np.array_equal(szo.decompress(s).view(np.uint32), rec.view(np.uint32))


@pytest.mark.parametrize("n", [1, 2])
def test_hyperplane_order_same_bytes(n):
    # every neighbour of a point has a smaller coordinate sum, so the order
    # by hyperplane yields the same recorded values and the same stream
    x = _field4((4, 5, 6, 7), seed=5)
    a = szo.compress(x, eb_rel=1e-3, n=n, m=8, order=0)
    b = szo.compress(x, eb_rel=1e-3, n=n, m=8, order=1)
    assert np.array_equal(a, b)


@pytest.mark.parametrize("n", [1, 2, 3, 4])
def test_unit_slowest_extent_is_the_3d_stream(n):
    # with one hyperplane along the slowest axis, every term reaching into it
    # reads 0 and adds exactly nothing: codes, recorded values and payload are
    # the 3D field's; the header differs in ndim and the stored 4th extent
    rng = np.random.default_rng(n)
    x3 = np.cumsum(np.cumsum(rng.normal(size=(6, 7, 9)), 1), 2).astype(np.float32)
    s3, r3, c3 = szo.compress(x3, eb_rel=1e-3, n=n, m=0, want_aux=True)
    s4, r4, c4 = szo.compress(x3[None], eb_rel=1e-3, n=n, m=0, want_aux=True)
    assert np.array_equal(c3, c4[0]) and np.array_equal(r3.view(np.uint32), r4[0].view(np.uint32))
    assert len(s3) == len(s4) and np.array_equal(s3[128:], s4[128:])
    assert set(np.nonzero(s3[:128] != s4[:128])[0].tolist()) == {8, 120}


@pytest.mark.parametrize("n", [1, 2, 3, 4])
def test_constant_hits_closed_form_4d(n):
    # exactly the n^4 corner points miss on a constant field (the partial
    # alternating binomial sums vanish once one index reaches n)
    x = np.full((5, 5, 6, 4), 1.0, np.float32)
    assert hitrate.hit_count(x, x, n, 0.5) == x.size - n ** 4


def test_invalid_and_corrupt():
    x = _field4((3, 4, 5, 6), seed=2)
    with pytest.raises(ValueError):
        szo.compress(x[None], eb_rel=1e-3)                      # 5D
    with pytest.raises(RuntimeError):
        szo.compress_lattice(x, eb_rel=1e-3)                    # the lattice form is 1D..3D
    s = szo.compress(x, eb_rel=1e-3, n=1, m=8).copy()
    s[120:128] = 0                                              # no 4th extent
    assert szo.decompress_rc(s) == szo.ECORRUPT
