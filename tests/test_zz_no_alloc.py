"""szgb_decompress_noalloc: the decompression entry point for callers that
cannot allocate device memory (a service with a fixed memory plan, code
running inside an allocator callback).  Its scratch is a fixed static device
array, so these tests check that its output equals szgb_decompress's and the
oracle's, bit for bit, on two calls in a row (the array keeps the previous
call's contents), across fields of every kind it decodes (1D-3D on the
wavefront, 3D with n = 3 and 4D on the hyperplane kernels), and that a
stream needing more scratch than the array holds is refused up front."""
import struct

import numpy as np
import pytest

from synthetic import fields

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    from paper_1706_03791_gb300 import build
    build.build()
    from paper_1706_03791_gb300 import szgb
    ctx = szgb.Context(0)
    yield torch, szgb, ctx
    ctx.close()


def _same(a, b):
    return np.array_equal(a.cpu().numpy().view(np.uint32), b.cpu().numpy().view(np.uint32))


CASES = [
    ("3d-n1", lambda: fields.blobs3d(24, 70, 44, seed=61, nblobs=6), dict(eb_rel=1e-4, m=0)),
    ("2d-n2", lambda: fields.grf2d(300, 130, seed=62), dict(eb_rel=1e-4, m=0, layers=2)),
    ("1d-n1", lambda: fields.grf2d(1, 3001, seed=63).reshape(3001), dict(eb_rel=1e-4, m=0)),
    ("2d-n4", lambda: fields.grf2d(97, 211, seed=64), dict(eb_rel=1e-4, m=0, layers=4)),
    ("3d-n3", lambda: fields.blobs3d(9, 30, 26, seed=65, nblobs=4), dict(eb_rel=1e-4, m=0, layers=3)),
    ("4d-n2", lambda: fields.blobs3d(12, 14, 20, seed=66, nblobs=4).reshape(3, 4, 14, 20),
     dict(eb_rel=1e-4, m=0, layers=2)),
]


@pytest.mark.parametrize("name,gen,kw", CASES, ids=[c[0] for c in CASES])
def test_noalloc_matches_decompress_twice(env, szo, name, gen, kw):
    torch, szgb, ctx = env
    x = np.ascontiguousarray(gen())
    xd = torch.from_numpy(x).cuda()
    s, _ = ctx.compress(xd, **kw)
    s = s.clone()
    ref = ctx.decompress(s)
    torch.cuda.synchronize()
    # the oracle's reconstruction of the same stream, independent of the GPU path
    rec = szo.decompress(s.cpu().numpy())
    assert np.array_equal(ref.cpu().numpy().reshape(-1).view(np.uint32),
                          np.ascontiguousarray(rec).reshape(-1).view(np.uint32))
    for _ in range(2):
        out = torch.full_like(ref, float("nan"))
        rc = szgb.decompress_noalloc(s, out, torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        assert rc == szgb.OK, szgb.strerror(rc)
        assert _same(out, ref)


def test_noalloc_refuses_unsupported(env, szo):
    """Streams this entry point does not decode are refused before any work:
    the lattice variant's."""
    torch, szgb, ctx = env
    cases = [
        szo.compress_lattice(fields.grf2d(40, 56, seed=73), eb_rel=1e-4, n=1, m=8),
    ]
    for sref in cases:
        s = torch.from_numpy(np.ascontiguousarray(sref)).cuda()
        out = torch.empty(8192, dtype=torch.float32, device="cuda")
        rc = szgb.decompress_noalloc(s, out, 0)
        assert rc == szgb.EUNSUPPORTED, szgb.strerror(rc)


def test_noalloc_refuses_oversize(env):
    torch, szgb, ctx = env
    # a consistent header for a 16 x 3200 x 10000 field with an empty payload:
    # its halo buffers alone exceed the fixed scratch
    d = (16, 3200, 10000)
    rows = d[0] * d[1]
    nsym, tw = 1, 2
    h = bytearray(128)
    h[0:4] = b"SZGB"
    struct.pack_into("<HH", h, 4, 1, 128)
    h[8], h[9], h[10], h[11], h[12], h[13] = 3, 1, 8, 1, 1, tw
    struct.pack_into("<3Q", h, 16, *d)
    struct.pack_into("<I", h, 68, nsym)
    cb = (3 * nsym + 3) & ~3
    tb = (tw * rows + 3) & ~3
    total = 128 + cb + tb
    struct.pack_into("<4Q", h, 72, rows, 0, 0, total)
    buf = np.zeros(total, np.uint8)
    buf[:128] = np.frombuffer(bytes(h), np.uint8)
    buf[128:131] = [128, 0, 1]
    s = torch.from_numpy(buf).cuda()
    out = torch.empty(16, dtype=torch.float32, device="cuda")
    rc = szgb.decompress_noalloc(s, out, 0)
    assert rc == szgb.ESCRATCH
