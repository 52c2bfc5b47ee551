"""Host-side checks of the C-ABI library (no GPU needed): it builds, loads,
exports every entry point include/szgb.h declares, and its host-only calls
(bound, header parsing, error strings) behave."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from conftest import ROOT


@pytest.fixture(scope="module")
def szgb():
    from paper_1706_03791_gb300 import build
    build.build()
    from paper_1706_03791_gb300 import szgb as m
    return m


def _declared():
    src = open(os.path.join(ROOT, "include", "szgb.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(szgb_[a-z0-9_]+)\s*\(", src)))


def test_exports_every_declared_symbol(szgb):
    lib = C.CDLL(szgb.LIB_PATH)
    names = _declared()
    assert len(names) >= 12
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(szgb.EXPORTS) == names


def test_strerror_and_bound(szgb):
    assert szgb.strerror(0) == "ok"
    assert "corrupt" in szgb.strerror(szgb.ECORRUPT)
    b = szgb.compress_bound((100, 500, 500))
    assert b > 100 * 500 * 500 * 4
    assert szgb.compress_bound((0, 5)) == 0


def test_stream_info_parses_oracle_header(szgb, szo):
    from synthetic import fields
    x = fields.blobs3d(6, 10, 12, seed=3, nblobs=3)
    s = szo.compress(x, eb_rel=1e-4, m=0)
    info = szgb.stream_info(s)
    h = szo.header(s)
    assert info["shape"] == x.shape and info["m"] == h["m"] and info["n_unpred"] == h["K"]
    bad = s.copy()
    bad[0] = 0
    with pytest.raises(szgb.SzgbError):
        szgb.stream_info(bad)
    with pytest.raises(szgb.SzgbError):
        szgb.stream_info(s[:-1])


def test_4d_stream_info(szgb, szo):
    # the oracle writes 4D streams (the predictor of Sec. III in four
    # dimensions); the library's header parser reads their four extents, and
    # declines a 4D header whose D x P reaches 2^32
    x = np.random.default_rng(4).normal(size=(3, 4, 5, 6)).astype(np.float32)
    s = szo.compress(x, eb_rel=1e-3, m=8)
    info = szgb.stream_info(s)
    assert info["ndim"] == 4 and info["shape"] == (3, 4, 5, 6)
    bad = s.copy()
    bad[120:128] = np.frombuffer(np.uint64(1 << 31).tobytes(), np.uint8)
    with pytest.raises(szgb.SzgbError) as e:
        szgb.stream_info(bad)
    assert e.value.code == szgb.ECORRUPT


def test_header_parser_survives_corruption(szgb, szo):
    # the library's host-side header check (szgb_stream_info) on mutated and
    # truncated headers: a parsed result or an error code, never a crash, and
    # a parsed shape always has ndim extents within the declared bounds
    x = np.random.default_rng(9).normal(size=(5, 7, 9)).astype(np.float32)
    s = szo.compress(x, eb_rel=1e-3, m=8)
    rng = np.random.default_rng(10)
    ok = 0
    for t in range(3000):
        m = s.copy()
        for _ in range(int(rng.integers(1, 4))):
            m[int(rng.integers(0, 128))] = int(rng.integers(0, 256))
        cut = int(rng.integers(0, len(m) + 1)) if t % 7 == 0 else len(m)
        try:
            info = szgb.stream_info(m[:cut])
        except szgb.SzgbError as e:
            assert e.code in (szgb.ECORRUPT, szgb.EUNSUPPORTED)
            continue
        ok += 1
        assert 1 <= info["ndim"] <= 3 and all(1 <= d < 2 ** 32 for d in info["shape"])
        assert 1 <= info["layers"] <= 4 and 2 <= info["m"] <= 16
    assert ok > 0


def test_suggest_m_matches_oracle(szgb, szo):
    # Algorithm 1's last step on the host: the library's suggestion from a
    # compression's counts equals the oracle's from its codes
    from oracle.hitrate import interval_hit_rate, suggest_m
    from synthetic import fields
    x = fields.grf2d(48, 40, seed=12)
    for m in (2, 3, 6, 10):
        for theta in (0.5, 0.9, 0.99, 1.0):
            s, _, codes = szo.compress(x, eb_rel=1e-4, m=m, want_aux=True)
            h = szo.header(s)
            st = szgb.Stats()
            st.n_points, st.n_unpred, st.m = x.size, h["K"], h["m"]
            got_m, got_r = szgb.suggest_m(st, theta)
            assert got_r == interval_hit_rate(codes)
            assert got_m == suggest_m(codes, m, theta)
    bad = szgb.Stats()
    bad.n_points, bad.n_unpred, bad.m = 10, 11, 8
    with pytest.raises(szgb.SzgbError):
        szgb.suggest_m(bad, 0.9)


@pytest.mark.gpu
def test_batch_parameters_checked_before_any_work(szgb):
    # every field's parameters and buffers are checked before the batch touches
    # any buffer: a bad field fails the whole call with SZGB_EINVAL (the
    # pointers here are not device memory; no kernel may run on them)
    L = szgb.lib()
    h = C.c_void_p()
    assert L.szgb_create(C.byref(h), 0, 0) == szgb.OK
    try:
        n = 2
        P = (szgb.Params * n)()
        P[0] = szgb.make_params((8, 8), eb_rel=1e-3)
        P[1] = szgb.make_params((2, 3, 4, 5), eb_rel=1e-3, m=1)  # m = 1: invalid
        dp = (C.c_void_p * n)(4096, 8192)
        op = (C.c_void_p * n)(4096 * 3, 4096 * 4)
        cap = (C.c_size_t * n)(1 << 16, 1 << 16)
        olen = (C.c_size_t * n)()
        assert L.szgb_compress_batch(h, n, dp, P, op, cap, olen, None) == szgb.EINVAL
        P[1] = szgb.make_params((2, 3, 4, 5), eb_rel=1e-3)
        dp[1] = 8200  # not 16-byte aligned
        assert L.szgb_compress_batch(h, n, dp, P, op, cap, olen, None) == szgb.EINVAL
        assert L.szgb_compress_batch(h, 0, dp, P, op, cap, olen, None) == szgb.EINVAL
        assert L.szgb_set_wave_ctas(h, -1) == szgb.EINVAL
        assert L.szgb_set_wave_ctas(h, 7) == szgb.OK
    finally:
        L.szgb_destroy(h)
