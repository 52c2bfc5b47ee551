"""Seeded synthetic FP32 fields standing in for the paper's datasets.

The paper evaluates on ATM climate fields (2D, 1800x3600), APS X-ray images
(2D, 2560x2560) and a Hurricane simulation (3D, 100x500x500) (Table 3).  None
of those datasets is available here, so every workload is generated from a
seed with the shapes of those datasets and smooth, spectrally-shaped values.

This module holds no part of the compression method: it only produces input
arrays.  Both the CPU oracle tests and the GPU path draw their inputs from it,
so the two sides always see identical bytes (``sha256`` records them).
"""
from __future__ import annotations

import hashlib
import os

import numpy as np


try:  # multithreaded FFTs (the same transform as numpy.fft)
    import scipy.fft as _fft
    _WORKERS = os.cpu_count() or 1
except ImportError:  # pragma: no cover
    _fft = None
    _WORKERS = 1


def sha256(a: np.ndarray) -> str:
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


def _spectral_noise(rng: np.random.Generator, shape, slope: float) -> np.ndarray:
    """Gaussian random field whose power spectrum falls as |k|^-slope.

    White N(0,1) noise is transformed to Fourier space, every mode is scaled
    by |k|^(-slope/2) (k=0 removed) and transformed back.  Returns float64
    with zero mean and unit standard deviation.
    """
    white = rng.standard_normal(shape)
    f = _fft.rfftn(white, workers=_WORKERS)
    ks = [np.fft.fftfreq(s) for s in shape[:-1]] + [np.fft.rfftfreq(shape[-1])]
    k2 = np.zeros(f.shape, dtype=np.float64)
    for ax, k in enumerate(ks):
        sh = [1] * len(shape)
        sh[ax] = k.size
        k2 = k2 + (k.reshape(sh) * shape[ax]) ** 2
    k2.flat[0] = 1.0
    f *= k2 ** (-slope / 4.0)
    f.flat[0] = 0.0
    g = _fft.irfftn(f, s=shape, axes=tuple(range(len(shape))), workers=_WORKERS)
    g -= g.mean()
    sd = g.std()
    return g / sd if sd > 0 else g


def grf2d(n0: int = 256, n1: int = 256, seed: int = 1, slope: float = 3.0,
          noise: float = 1e-3) -> np.ndarray:
    """2D Gaussian random field, power ~ k^-slope, scaled to range 1, plus
    white noise N(0, noise * range).  The small-field workload (256x256,
    k^-3, noise 1e-3 of the range)."""
    rng = np.random.default_rng(seed)
    g = _spectral_noise(rng, (n0, n1), slope)
    g = (g - g.min()) / (g.max() - g.min())
    g = g + rng.standard_normal(g.shape) * noise
    return g.astype(np.float32)


def blobs3d(n0: int = 100, n1: int = 500, n2: int = 500, seed: int = 2,
            nblobs: int = 64, turb: float = 0.1) -> np.ndarray:
    """3D smooth field: a sum of Gaussian blobs (centres uniform, sigma
    log-uniform in [5, 40] cells, amplitudes N(0,1)) plus k^-11/3 turbulence
    scaled to `turb` of the blob field's standard deviation.  Stands in for
    the 100x500x500 Hurricane fields."""
    rng = np.random.default_rng(seed)
    shape = (n0, n1, n2)
    f = np.zeros(shape, dtype=np.float64)
    ax = [np.arange(s, dtype=np.float64) for s in shape]
    for _ in range(nblobs):
        c = [rng.uniform(0, s) for s in shape]
        sig = float(np.exp(rng.uniform(np.log(5.0), np.log(40.0))))
        amp = rng.standard_normal()
        g = [np.exp(-0.5 * ((a - cc) / sig) ** 2) for a, cc in zip(ax, c)]
        f += amp * (g[0][:, None, None] * g[1][None, :, None]) * g[2][None, None, :]
    t = _spectral_noise(rng, shape, 11.0 / 3.0)
    sd = f.std()
    f += t * (turb * (sd if sd > 0 else 1.0))
    return f.astype(np.float32)


def climate2d(seed: int, n0: int = 1800, n1: int = 3600, mask: bool = False,
              front: bool = False) -> np.ndarray:
    """Climate-like 2D field: a latitude profile (cosine series with random
    coefficients) plus a random field with spectral slope drawn from
    U[2, 4].  Optionally a constant masked region (~30% of the area set to
    the field minimum) or a sharp step front (jump of 0.2 of the range
    along a random curve).  Stands in for one 1800x3600 ATM field."""
    rng = np.random.default_rng(seed)
    lat = np.linspace(-np.pi / 2, np.pi / 2, n0)
    prof = np.zeros(n0)
    for h in range(1, 6):
        prof += rng.standard_normal() / h * np.cos(h * lat + rng.uniform(0, np.pi))
    slope = rng.uniform(2.0, 4.0)
    g = _spectral_noise(rng, (n0, n1), slope)
    f = prof[:, None] * 2.0 + 0.5 * g
    rngv = f.max() - f.min()
    if front:
        cols = np.arange(n1)
        a = rng.uniform(0.2, 0.8) * n0
        b = rng.uniform(0.02, 0.1) * n0
        ph = rng.uniform(0, 2 * np.pi)
        curve = a + b * np.sin(2 * np.pi * cols / n1 * rng.integers(1, 4) + ph)
        rows = np.arange(n0)[:, None]
        f = f + 0.2 * rngv * (rows > curve[None, :])
    if mask:
        lo = f.min()
        m = _spectral_noise(rng, (n0, n1), 4.0)
        thr = np.quantile(m, 0.7)
        f = np.where(m > thr, lo, f)
    return f.astype(np.float32)


def climate_batch_field(i: int, nfields: int = 79, n0: int = 1800, n1: int = 3600,
                        seed0: int = 300) -> np.ndarray:
    """Field i of the climate batch: seed seed0 + i; 15% of the fields
    (12 of 79) carry a masked constant region and 5% (4 of 79) a step
    front, spread evenly over the batch."""
    nmask = round(0.15 * nfields)
    nfront = round(0.05 * nfields)
    masked = {(k * nfields) // max(nmask, 1) + 1 for k in range(nmask)}
    fronts = {(k * nfields) // max(nfront, 1) + 3 for k in range(nfront)}
    return climate2d(seed0 + i, n0, n1, mask=i in masked, front=i in fronts)


def climate_batch(nfields: int = 79, n0: int = 1800, n1: int = 3600,
                  seed0: int = 300) -> list:
    """The 79-field climate batch (climate_batch_field for i = 0..78)."""
    return [climate_batch_field(i, nfields, n0, n1, seed0) for i in range(nfields)]


def uneven_batch(nfields: int = 512, seed: int = 4, seed0: int = 4000,
                 side2=(64, 2048), side3=(32, 256), ebs=(1e-3, 1e-4, 1e-5)) -> list:
    """The uneven batch: half 2D fields with side log-uniform in side2, half
    3D fields with side log-uniform in side3 (sizes and bounds drawn from
    `seed`), each a k^-3 Gaussian random field scaled to range 1 (field i
    from seed seed0 + i), with a value-range-relative bound drawn from
    `ebs`.  Returns a list of (array, eb_rel)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(nfields):
        if i % 2 == 0:
            n = int(round(np.exp(rng.uniform(np.log(side2[0]), np.log(side2[1])))))
            shape = (n, n)
        else:
            n = int(round(np.exp(rng.uniform(np.log(side3[0]), np.log(side3[1])))))
            shape = (n, n, n)
        eb = float(ebs[int(rng.integers(0, len(ebs)))])
        g = _spectral_noise(np.random.default_rng(seed0 + i), shape, 3.0)
        g = (g - g.min()) / max(g.max() - g.min(), 1e-30)
        out.append((g.astype(np.float32), eb))
    return out


def linear_field(shape, coef=(0.5, -0.25, 0.125), c0=1.0) -> np.ndarray:
    """Dyadic linear field c0 + sum_a coef[a] * index_a (exact in float32)."""
    grids = np.meshgrid(*[np.arange(s, dtype=np.float64) for s in shape], indexing="ij")
    f = np.full(shape, c0, dtype=np.float64)
    for a, gi in enumerate(grids):
        f = f + coef[a] * gi
    return f.astype(np.float32)


def walk3d(n0: int, n1: int, n2: int, seed: int, step: float = 0.01) -> np.ndarray:
    """Seeded random walk along the fastest axis, in [0, 1]: a cheap field of
    any shape (many short rows without a spectral transform)."""
    rng = np.random.default_rng(seed)
    g = np.cumsum(rng.standard_normal((n0, n1, n2), dtype=np.float32) * np.float32(step), axis=2)
    g += rng.standard_normal((n0, n1, 1), dtype=np.float32)
    g -= g.min()
    g /= max(float(g.max()), 1e-30)
    return np.ascontiguousarray(g, dtype=np.float32)


def cache_dir() -> str:
    d = os.environ.get("SZGB_SYNTH_CACHE") or os.path.join(
        os.environ.get("TMPDIR", "/tmp"), "szgb_synth")
    os.makedirs(d, exist_ok=True)
    return d


def cached(name: str, fn, *args, **kw) -> np.ndarray:
    """Generate once per machine and keep the bytes in a local cache."""
    p = os.path.join(cache_dir(), name + ".npy")
    if os.path.exists(p):
        try:
            return np.load(p)
        except Exception:
            pass
    a = fn(*args, **kw)
    tmp = p + ".%d.tmp.npy" % os.getpid()
    np.save(tmp, a)
    os.replace(tmp, p)
    return a


def workload_small() -> np.ndarray:
    """2D 256x256 k^-3 field with 1e-3 noise (seed 1)."""
    return cached("grf2d_256_s1", grf2d, 256, 256, 1)


def workload_3d() -> np.ndarray:
    """3D 100x500x500 blob + turbulence field (seed 2)."""
    return cached("blobs3d_100x500x500_s2", blobs3d, 100, 500, 500, 2)
