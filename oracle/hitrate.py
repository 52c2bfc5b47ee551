"""Prediction hitting rate (Sec. III) and the best-layer comparison of Table 2,
plain NumPy on top of the oracle's predictor and compressor.

TEST INFRASTRUCTURE ONLY: imported by the tests and run as a report
(``python -m oracle.hitrate``); the product counts the same hits on the
device in ``szgb_hit_count_dev``.

Definitions (Sec. III): a point is predictable when its original value and
its n-layer prediction differ by no more than the error bound; the hitting
rate R_PH = N_PH / N is the share of such points.  R_PH^orig predicts every
point from the ORIGINAL values of its preceding neighbours, R_PH^decomp from
the values the compressor recorded for them (the decompressed values), which
is the prediction the compressor actually makes.

Readings where the passage leaves a detail open:
  * "not larger than" is inclusive: hit <=> |x_i - f_i| <= eb.
  * the prediction f_i is the float32 value the compressor forms (the oracle's
    predictor: terms in descending lexicographic order, values outside the
    domain 0); the difference and the comparison are taken in float64 of the
    float32 values, so the decision has no rounding of its own.
  * eb is the compressor's effective float32 bound eb_f for the field, and
    R_PH^decomp is taken from a compression with the same layer count, bound
    and interval count m (the recorded values of quantized and unpredictable
    points depend on m).
  * the quantizer's centre code (q = 0) implies a hit, since it needs
    |x - f| < eb_f; a hit without the centre code only happens when |x - f|
    lies within rounding of eb_f.
"""
from __future__ import annotations

import numpy as np

from . import szo


def hit_count(x, v, n: int, eb: float) -> int:
    """Number of points of x whose n-layer prediction from the values v at
    the preceding neighbours lies within eb of x (v = x: original values)."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    v = np.ascontiguousarray(v, dtype=np.float32)
    if x.shape != v.shape:
        raise ValueError("x and v need the same shape")
    f = szo.predict_field(v, n)
    return int(np.count_nonzero(np.abs(x.astype(np.float64) - f.astype(np.float64)) <= eb))


def hit_rates(x, n: int, mode=szo.REL, eb_abs=0.0, eb_rel=1e-4, m=0, theta=0.99) -> dict:
    """R_PH^orig and R_PH^decomp of x for the n-layer predictor under the
    given bound, with the compressor's own recorded values for the latter."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    stream, rec, codes = szo.compress(x, mode=mode, eb_abs=eb_abs, eb_rel=eb_rel, n=n, m=m,
                                      theta=theta, want_aux=True)
    hdr = szo.header(stream)
    eb_f, m_used = hdr["eb_f"], hdr["m"]
    N = x.size
    h_orig = hit_count(x, x, n, eb_f)
    h_dec = hit_count(x, rec, n, eb_f)
    return {"n": n, "N": N, "eb_f": eb_f, "m": m_used, "hits_orig": h_orig, "hits_decomp": h_dec,
            "R_orig": h_orig / N, "R_decomp": h_dec / N, "rec": rec, "codes": codes}


def interval_hit_rate(codes) -> float:
    """Algorithm 1, counting step after the coding (Sec. IV-B): the share of
    points that fell into one of the 2^m - 1 quantization intervals, i.e.
    whose code is not the unpredictable code 0."""
    codes = np.asarray(codes)
    return float(np.count_nonzero(codes != 0)) / codes.size


def suggest_m(codes, m: int, theta: float) -> int:
    """Algorithm 1, last step (Sec. IV-B): when the interval hit rate stays
    below theta a larger m is suggested (m + 1, at most 16); otherwise m."""
    if interval_hit_rate(codes) < theta:
        return min(m + 1, 16)
    return m


def best_layer_table(x, layers=(1, 2, 3, 4), **kw) -> list:
    """One row per layer count, as in Table 2: (n, R_PH^orig, R_PH^decomp, m)."""
    rows = []
    for n in layers:
        r = hit_rates(x, n, **kw)
        rows.append((n, r["R_orig"], r["R_decomp"], r["m"]))
    return rows


def _report():
    from synthetic import fields
    cases = [
        ("2D 512x512 k^-6 field, no noise", fields.grf2d(512, 512, seed=3, slope=6.0, noise=0.0)),
        ("2D 256x256 k^-3 field + 1e-3 noise", fields.grf2d(256, 256, seed=1)),
        ("3D 64^3 blobs, no turbulence", fields.blobs3d(64, 64, 64, seed=2, turb=0.0)),
        ("3D 64^3 blobs + 1% turbulence", fields.blobs3d(64, 64, 64, seed=2, turb=0.01)),
    ]
    for eb_rel in (1e-3, 1e-4):
        for name, x in cases:
            print("%s, rel eb %g" % (name, eb_rel))
            print("  n   R_PH^orig   R_PH^decomp   m")
            for n, ro, rd, m in best_layer_table(x, (1, 2, 3, 4), eb_rel=eb_rel):
                print("  %d   %8.4f%%   %8.4f%%   %d" % (n, 100 * ro, 100 * rd, m))


if __name__ == "__main__":
    _report()
