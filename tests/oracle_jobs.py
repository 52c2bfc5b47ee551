"""Oracle work for the full-size parity tests, run in spawned worker
processes (one field per task).  TEST INFRASTRUCTURE: it calls only the CPU
oracle and the seeded input generators.

Each job regenerates its field from its seed (so only the seed crosses the
process boundary on the way in), compresses it with the oracle, and returns
the field, the oracle's stream and the SHA-256 of the oracle's recorded
(decompressed) values, which the GPU reconstruction must equal bit for bit.
"""
from __future__ import annotations

import hashlib

import numpy as np


def field(kind: str, idx: int):
    """(array, keyword arguments of the compression) of field `idx` of a
    workload."""
    from synthetic import fields
    if kind == "climate79":
        # fields.climate_batch() field by field: seeds 300..378, 12 masked, 4 fronts
        return fields.climate_batch_field(idx), dict(eb_rel=1e-4, m=0)
    if kind == "uneven512":
        shape, eb = uneven_shape(idx)
        g = fields._spectral_noise(np.random.default_rng(4000 + idx), shape, 3.0)
        g = (g - g.min()) / max(g.max() - g.min(), 1e-30)
        return g.astype(np.float32), dict(eb_rel=eb, m=0)
    if kind == "serve":
        shape = serve_shape(idx)
        g = fields._spectral_noise(np.random.default_rng(5000 + idx), shape, 3.0)
        g = (g - g.min()) / max(g.max() - g.min(), 1e-30)
        return g.astype(np.float32), dict(eb_rel=1e-4, m=0)
    raise ValueError(kind)


def uneven_shape(idx: int):
    """Shape and bound of field idx of fields.uneven_batch() (same draws)."""
    rng = np.random.default_rng(4)
    for i in range(idx + 1):
        if i % 2 == 0:
            n = int(round(np.exp(rng.uniform(np.log(64), np.log(2048)))))
            shape = (n, n)
        else:
            n = int(round(np.exp(rng.uniform(np.log(32), np.log(256)))))
            shape = (n, n, n)
        eb = float((1e-3, 1e-4, 1e-5)[int(rng.integers(0, 3))])
    return shape, eb


def serve_shape(idx: int):
    """Request idx of the serving recipe: even requests 2D with side
    log-uniform in [256, 4096], odd ones 3D with side log-uniform in
    [64, 512] (seed 55)."""
    rng = np.random.default_rng(55)
    for i in range(idx + 1):
        if i % 2 == 0:
            n = int(round(np.exp(rng.uniform(np.log(256), np.log(4096)))))
            shape = (n, n)
        else:
            n = int(round(np.exp(rng.uniform(np.log(64), np.log(512)))))
            shape = (n, n, n)
    return shape


def rec_sha(a) -> str:
    return hashlib.sha256(np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).tobytes()).hexdigest()


def job(args):
    """(idx, field or None, oracle stream, SHA-256 of the recorded values);
    args = (kind, idx, want_x[, chunk_points])."""
    kind, idx, want_x = args[:3]
    chunk = args[3] if len(args) > 3 else 0
    from oracle import szo
    x, kw = field(kind, idx)
    s, rec, _ = szo.compress(x, want_aux=True, chunk_points=chunk, **kw)
    return idx, (x if want_x else None), s, rec_sha(rec)


def gen(args):
    """(idx, field) without the oracle."""
    kind, idx = args
    return idx, field(kind, idx)[0]


def noop(_):
    return 0
