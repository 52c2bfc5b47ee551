"""Parity on the benchmark workloads at their full sizes and with their own
generators: every stream byte-identical to the CPU oracle's and every
reconstruction bit-identical to the values the oracle recorded.

  * 79 climate-like 1800 x 3600 fields (12 with constant masked regions, 4
    with step fronts), rel eb 1e-4, adaptive m: one batched call (captured,
    then replayed from its CUDA graph) and one call per field;
  * 512 uneven fields (2D 64^2..2048^2, 3D 32^3..256^3, rel eb 1e-3/1e-4/1e-5)
    in one batched call with the autotuned wavefront shape, replayed;
  * the 3D 100 x 500 x 500 field at rel eb 1e-6 with n = 1 and n = 2;
  * 16 served requests drawn from the serving recipe (2D 256^2..4096^2, 3D
    64^3..512^3, k^-3 fields, rel eb 1e-4), half compress and half
    decompress, through the server under a 100 GB budget.

The oracle runs in a spawned process pool, one field per task, started
before the first GPU call; reconstructions are compared through SHA-256 of
their bits (a mismatch names the field)."""
import multiprocessing as mp
import os
import time

import numpy as np
import pytest

import oracle_jobs as J

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pool():
    from oracle import szo
    szo.build()
    n = max(1, min(32, os.cpu_count() or 1))
    p = mp.get_context("spawn").Pool(n)
    p.map(J.noop, range(n), chunksize=1)  # start the workers now
    yield p
    p.close()
    p.join()


@pytest.fixture(scope="module")
def env(pool):
    import torch
    from paper_1706_03791_gb300 import build
    build.build()
    from paper_1706_03791_gb300 import szgb
    c = szgb.Context(0)
    yield torch, szgb, c
    c.close()


def _oracle(pool, kind, idxs, want_x=True, chunk=0):
    out = {}
    for idx, x, s, h in pool.imap_unordered(J.job, [(kind, i, want_x, chunk) for i in idxs], chunksize=1):
        out[idx] = (x, s, h)
    return [out[i] for i in idxs]


def _check_streams(streams, refs, what):
    for i, (s, (_, sref, _)) in enumerate(zip(streams, refs)):
        sg = s.cpu().numpy()
        assert sg.size == sref.size and np.array_equal(sg, sref), "%s field %d: stream differs" % (what, i)


def _check_recon(ys, refs, what):
    for i, (y, (_, _, h)) in enumerate(zip(ys, refs)):
        assert J.rec_sha(y.cpu().numpy()) == h, "%s field %d: reconstruction differs" % (what, i)


def test_climate79_batched_and_per_field(env, pool):
    torch, szgb, ctx = env
    t0 = time.perf_counter()
    refs = _oracle(pool, "climate79", range(79))
    kw = dict(eb_rel=1e-4, m=0)
    xs = [torch.from_numpy(x).cuda() for x, _, _ in refs]
    for rep in range(2):  # captured, then replayed
        sb, st = ctx.compress_batch(xs, kw)
        _check_streams(sb, refs, "batched #%d" % rep)
        ys = ctx.decompress_batch(sb)
        _check_recon(ys, refs, "batched #%d" % rep)
        del ys
    for i, x in enumerate(xs):  # one call per field
        s, _ = ctx.compress(x, **kw)
        _check_streams([s], [refs[i]], "single %d" % i)
        _check_recon([ctx.decompress(s)], [refs[i]], "single %d" % i)
    print("climate79: %.1f s" % (time.perf_counter() - t0))


def test_uneven512_autotuned_graph(env, pool):
    """The autotuner picks the wavefront shape and the Huffman chunk length;
    the oracle then codes every field with that chunk length."""
    torch, szgb, ctx = env
    t0 = time.perf_counter()
    gen = dict(pool.imap_unordered(J.gen, [("uneven512", i) for i in range(512)], chunksize=1))
    kws = [dict(eb_rel=J.uneven_shape(i)[1], m=0) for i in range(512)]
    xs = [torch.from_numpy(gen[i]).cuda() for i in range(512)]
    del gen
    tuned = ctx.autotune_batch(xs, kws, reps=1)
    assert tuned["W"] >= 1
    chunk = 0 if tuned["chunk"] == szgb.CHUNK_ROWS else tuned["chunk"]
    refs = _oracle(pool, "uneven512", range(512), want_x=False, chunk=chunk)
    for rep in range(2):  # captured with the tuned shape and chunking, then replayed
        sb, st = ctx.compress_batch(xs, kws)
        _check_streams(sb, refs, "uneven #%d" % rep)
        ys = ctx.decompress_batch(sb)
        _check_recon(ys, refs, "uneven #%d" % rep)
        del ys
    print("uneven512: %.1f s (W = %d, chunk %d)" % (time.perf_counter() - t0, tuned["W"], chunk))


@pytest.mark.parametrize("layers", [1, 2])
def test_3d_field_rel_1e6(env, layers):
    torch, szgb, ctx = env
    from oracle import szo
    from synthetic import fields
    x = fields.workload_3d()
    kw = dict(eb_rel=1e-6, m=0, layers=layers)
    sref, rec, _ = szo.compress(x, want_aux=True, **kw)
    xd = torch.from_numpy(x).cuda()
    for _ in range(2):
        s, st = ctx.compress(xd, **kw)
        assert np.array_equal(s.cpu().numpy(), sref)
        y = ctx.decompress(s)
        assert np.array_equal(y.cpu().numpy().view(np.uint32), rec.view(np.uint32))


def test_served_requests(env, pool):
    torch, szgb, ctx = env
    t0 = time.perf_counter()
    n = 16
    refs = _oracle(pool, "serve", range(n))
    srv = szgb.Server(0, budget=100 << 30, workers=3, max_batch=32)
    try:
        tickets = []
        for i, (x, sref, h) in enumerate(refs):
            if i % 4 < 2:  # compress requests
                out = np.empty(x.size * 4 + (1 << 16), np.uint8)
                tickets.append((i, "c", out, srv.submit_compress(x, out, eb_rel=1e-4, m=0)))
            else:  # decompress requests of the oracle's streams
                out = np.empty(x.shape, np.float32)
                tickets.append((i, "d", out, srv.submit_decompress(sref, out)))
        for i, op, out, t in tickets:
            st, nbytes = srv.wait(t)
            assert st == 0, (i, szgb.strerror(st))
            _, sref, h = refs[i]
            if op == "c":
                assert nbytes == sref.size and np.array_equal(out[:nbytes], sref), "request %d: stream" % i
            else:
                assert J.rec_sha(out) == h, "request %d: reconstruction" % i
    finally:
        srv.close()
    print("served: %.1f s" % (time.perf_counter() - t0))
