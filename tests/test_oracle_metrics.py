"""The oracle's quality metrics (Sec. II, Metrics 1-4) pinned to closed forms
and a small example worked by hand."""
import math

import numpy as np
import pytest

from oracle.metrics import bit_rate, compression_factor, quality


def test_exact_reconstruction():
    x = np.linspace(-2.0, 5.0, 101)
    q = quality(x, x.copy())
    assert q["rmse"] == 0.0 and q["max_abs_err"] == 0.0 and q["nrmse"] == 0.0
    assert q["psnr"] == math.inf
    assert q["pearson"] == pytest.approx(1.0, abs=1e-15)


def test_constant_offset():
    # e_i = -c for every point: RMSE = max error = |c|, the shape is unchanged
    rng = np.random.default_rng(3)
    x = rng.normal(size=1000)
    c = 0.125
    q = quality(x, x + c)
    rx = x.max() - x.min()
    assert q["rmse"] == pytest.approx(c, rel=1e-12)
    assert q["max_abs_err"] == pytest.approx(c, rel=1e-12)
    assert q["nrmse"] == pytest.approx(c / rx, rel=1e-12)
    assert q["psnr"] == pytest.approx(20 * math.log10(rx / c), rel=1e-12)
    assert q["pearson"] == pytest.approx(1.0, abs=1e-12)


def test_negated_and_scaled():
    rng = np.random.default_rng(4)
    x = rng.uniform(-1, 3, size=500)
    assert quality(x, -2.0 * x + 7.0)["pearson"] == pytest.approx(-1.0, abs=1e-12)
    assert quality(x, 0.5 * x)["pearson"] == pytest.approx(1.0, abs=1e-12)


def test_worked_example():
    # x = 0 1 2 3, y = 0 1 2 4: e = 0 0 0 -1, R_X = 3
    # rmse = sqrt(1/4) = 1/2, nrmse = 1/6, psnr = 20 log10 6
    # centred x: -1.5 -0.5 0.5 1.5; centred y (mean 7/4): -1.75 -0.75 0.25 2.25
    # sum xy = 6.5, sum xx = 5, sum yy = 8.75: rho = 6.5 / sqrt(43.75)
    q = quality([0, 1, 2, 3], [0, 1, 2, 4])
    assert q["rmse"] == pytest.approx(0.5, rel=1e-15)
    assert q["nrmse"] == pytest.approx(1 / 6, rel=1e-15)
    assert q["psnr"] == pytest.approx(20 * math.log10(6.0), rel=1e-15)
    assert q["max_abs_err"] == 1.0 and q["max_rel_err"] == pytest.approx(1 / 3, rel=1e-15)
    assert q["pearson"] == pytest.approx(6.5 / math.sqrt(43.75), rel=1e-14)


def test_undefined_cases():
    q = quality(np.full(10, 2.5), np.full(10, 2.5))
    assert q["psnr"] == math.inf and math.isnan(q["nrmse"]) and math.isnan(q["pearson"])
    q = quality(np.full(10, 2.5), np.full(10, 2.0))
    assert math.isnan(q["psnr"]) and q["rmse"] == pytest.approx(0.5)
    with pytest.raises(ValueError):
        quality([1.0, 2.0], [1.0])


def test_cf_br_relation():
    # BR * CF = 32 for binary32 data (Metric 4)
    for n, b in ((1000, 371), (25_000_000, 13_040_186)):
        assert bit_rate(n, b) * compression_factor(n, b) == pytest.approx(32.0, rel=1e-15)
