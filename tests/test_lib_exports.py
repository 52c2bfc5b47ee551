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
    return sorted(set(re.findall(r"\b(szgb_[a-z_]+)\s*\(", src)))


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


def test_4d_stream_reported_unsupported(szgb, szo):
    # the oracle writes 4D streams (the predictor of Sec. III in four
    # dimensions); the GPU library recognises and declines them
    x = np.random.default_rng(4).normal(size=(3, 4, 5, 6)).astype(np.float32)
    s = szo.compress(x, eb_rel=1e-3, m=8)
    with pytest.raises(szgb.SzgbError) as e:
        szgb.stream_info(s)
    assert e.value.code == szgb.EUNSUPPORTED
