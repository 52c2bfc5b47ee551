"""Reconstruction quality and size metrics (Sec. II, Metrics 1-4), plain NumPy
in float64.

TEST INFRASTRUCTURE ONLY: imported by the tests and the benchmark harness's
checks; the product computes the same figures in ``szgb_quality``.

Readings where the definitions leave a case open:
  * R_X is the value range of the original data, max(x) - min(x).
  * the standard deviations in Pearson's coefficient are population ones
    (divisor N), as is the covariance; the ratio does not depend on it.
  * R_X = 0 (a constant field) leaves NRMSE and PSNR undefined: NaN, except
    PSNR = +inf when the reconstruction is exact (RMSE = 0).  A zero standard
    deviation leaves the coefficient undefined: NaN.
"""
from __future__ import annotations

import math

import numpy as np


def quality(x, y) -> dict:
    """Metrics 1-3 of the reconstruction y of x (any shape, same size)."""
    x = np.asarray(x, dtype=np.float64).ravel()
    y = np.asarray(y, dtype=np.float64).ravel()
    if x.size != y.size or x.size == 0:
        raise ValueError("x and y need the same, nonzero size")
    n = x.size
    e = x - y                                   # Metric 1: e_abs_i = x_i - y_i
    rx = float(x.max() - x.min())               # R_X
    max_abs = float(np.abs(e).max())
    rmse = math.sqrt(float(np.sum(e * e)) / n)  # Metric 2
    nrmse = rmse / rx if rx > 0 else float("nan")
    if rmse == 0.0:
        psnr = float("inf")
    else:
        psnr = 20.0 * math.log10(rx / rmse) if rx > 0 else float("nan")
    xm, ym = x - x.mean(), y - y.mean()         # Metric 3
    sx = math.sqrt(float(np.sum(xm * xm)) / n)
    sy = math.sqrt(float(np.sum(ym * ym)) / n)
    cov = float(np.sum(xm * ym)) / n
    rho = cov / (sx * sy) if sx > 0 and sy > 0 else float("nan")
    return {"n": n, "x_min": float(x.min()), "x_max": float(x.max()), "max_abs_err": max_abs,
            "max_rel_err": max_abs / rx if rx > 0 else float("nan"), "rmse": rmse, "nrmse": nrmse,
            "psnr": psnr, "pearson": rho}


def compression_factor(n_values: int, stream_bytes: int, value_bytes: int = 4) -> float:
    """Metric 4: original size over compressed size."""
    return n_values * value_bytes / stream_bytes


def bit_rate(n_values: int, stream_bytes: int) -> float:
    """Metric 4: compressed bits per value (BR * CF = 32 for binary32 data)."""
    return stream_bytes * 8.0 / n_values
