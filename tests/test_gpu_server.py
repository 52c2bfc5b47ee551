"""The serving loop on the GPU: a mix of compress and decompress requests of
different shapes, submitted while earlier ones are on the device, under a
budget small enough that admission has to wait.  Every result is the result
of the field alone: compressed streams byte-identical to the oracle's,
reconstructions bit-identical."""
import numpy as np
import pytest

from synthetic import fields

pytestmark = pytest.mark.gpu


def _bits(a):
    return np.ascontiguousarray(a).view(np.uint32)


def test_server_mix(szo):
    from paper_1706_03791_gb300 import build
    build.build()
    from paper_1706_03791_gb300 import szgb
    gens = [
        (lambda: fields.grf2d(256, 256, seed=81), dict(eb_rel=1e-4, m=0)),
        (lambda: fields.blobs3d(20, 40, 44, seed=82, nblobs=8), dict(eb_rel=1e-4, m=0)),
        (lambda: fields.grf2d(300, 211, seed=83), dict(eb_rel=1e-3, layers=2, m=0)),
        (lambda: fields.grf2d(1, 3000, seed=84).reshape(3000), dict(eb_rel=1e-4, m=8)),
        (lambda: fields.blobs3d(9, 33, 20, seed=85, nblobs=4), dict(mode=0, eb_abs=1e-3, m=6)),
    ]
    xs = [np.ascontiguousarray(g()) for g, _ in gens]
    kws = [kw for _, kw in gens]
    refs = [szo.compress(x, want_aux=True, **kw) for x, kw in zip(xs, kws)]
    # budget for about two requests at a time
    srv = szgb.Server(0, budget=24 << 20, workers=2, max_batch=3)
    try:
        jobs = []
        for rep in range(3):
            for i, (x, kw) in enumerate(zip(xs, kws)):
                out = np.empty(x.nbytes * 2 + (1 << 16), np.uint8)
                jobs.append(("c", i, out, srv.submit_compress(x, out, **kw)))
                y = np.empty(x.shape, np.float32)
                jobs.append(("d", i, y, srv.submit_decompress(refs[i][0], y)))
        for kind, i, buf, t in jobs:
            st, n = srv.wait(t)
            assert st == 0, szgb.strerror(st)
            if kind == "c":
                assert n == refs[i][0].size and np.array_equal(buf[:n], refs[i][0]), "stream %d differs" % i
            else:
                assert np.array_equal(_bits(buf), _bits(refs[i][1])), "reconstruction %d differs" % i
        s = srv.stats()
        assert s["completed"] == len(jobs) and s["peak_reserved"] <= 24 << 20
    finally:
        srv.close()


def test_server_every_field_kind(szo):
    """Requests the batched wavefront does not carry (3D n = 3, 4D, the
    lattice variant) run alone on their own kernels, between batches of
    wavefront requests; every result equals the oracle's."""
    from paper_1706_03791_gb300 import build
    build.build()
    from paper_1706_03791_gb300 import szgb
    rng = np.random.default_rng(86)
    x4 = fields.blobs3d(12, 10, 24, seed=87, nblobs=4).reshape(3, 4, 10, 24) + \
        rng.normal(scale=1e-4, size=(3, 4, 10, 24)).astype(np.float32)
    cases = [
        (fields.blobs3d(8, 21, 26, seed=88, nblobs=4), dict(eb_rel=1e-4, layers=3, m=0), "exact"),
        (np.ascontiguousarray(x4, dtype=np.float32), dict(eb_rel=1e-4, layers=2, m=0), "exact"),
        (fields.grf2d(60, 70, seed=89), dict(eb_rel=1e-4, m=0, variant=1), "lattice"),
        (fields.grf2d(128, 96, seed=90), dict(eb_rel=1e-4, m=0), "exact"),
    ]
    refs = []
    for x, kw, kind in cases:
        if kind == "lattice":
            k = {a: b for a, b in kw.items() if a != "variant"}
            s, rec, _ = szo.compress_lattice(x, want_aux=True, **k)
        else:
            s, rec, _ = szo.compress(x, want_aux=True, **kw)
        refs.append((s, rec))
    srv = szgb.Server(0, budget=64 << 20, workers=2, max_batch=4)
    try:
        jobs = []
        for rep in range(2):
            for i, (x, kw, _) in enumerate(cases):
                out = np.empty(x.nbytes * 3 + (1 << 16), np.uint8)
                jobs.append(("c", i, out, srv.submit_compress(x, out, **kw)))
                y = np.empty(x.shape, np.float32)
                jobs.append(("d", i, y, srv.submit_decompress(refs[i][0], y)))
        for kind, i, buf, t in jobs:
            st, n = srv.wait(t)
            assert st == 0, szgb.strerror(st)
            if kind == "c":
                assert n == refs[i][0].size and np.array_equal(buf[:n], refs[i][0]), "stream %d differs" % i
            else:
                assert np.array_equal(_bits(buf), _bits(refs[i][1])), "reconstruction %d differs" % i
    finally:
        srv.close()
