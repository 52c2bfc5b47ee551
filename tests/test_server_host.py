"""Host-side behaviour of the serving loop (no GPU needed): argument checks,
budget admission, tickets, and that every request completes -- on a machine
without a GPU the workers cannot create a context and complete every request
with SZGB_ECUDA, which exercises the queue and completion path."""
import numpy as np
import pytest


@pytest.fixture(scope="module")
def szgb():
    from paper_1706_03791_gb300 import build
    build.build()
    from paper_1706_03791_gb300 import szgb as m
    return m


def _gpu():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


def test_server_arguments(szgb):
    import ctypes as C
    h = C.c_void_p()
    L = szgb.lib()
    assert L.szgb_server_create(C.byref(h), 0, 0, 1, 4) == szgb.EINVAL      # no budget
    assert L.szgb_server_create(C.byref(h), 0, 1 << 20, 0, 4) == szgb.EINVAL  # no worker
    assert L.szgb_server_create(C.byref(h), 0, 1 << 20, 1, 0) == szgb.EINVAL  # no batch


def test_server_budget_and_validation(szgb):
    srv = szgb.Server(0, budget=8 << 20, workers=1, max_batch=4)
    try:
        big = np.zeros((1024, 1024), np.float32)          # footprint > 8 MiB
        with pytest.raises(szgb.SzgbError) as e:
            srv.submit_compress(big, np.empty(1 << 20, np.uint8), eb_rel=1e-4)
        assert e.value.code == szgb.EBUDGET
        bad = np.zeros(100, np.uint8)                      # not a stream
        with pytest.raises(szgb.SzgbError) as e:
            srv.submit_decompress(bad, np.empty(10, np.float32))
        assert e.value.code == szgb.ECORRUPT
    finally:
        srv.close()


@pytest.mark.skipif(_gpu(), reason="checks the no-GPU completion path")
def test_server_completes_every_request_without_gpu(szgb):
    srv = szgb.Server(0, budget=64 << 20, workers=2, max_batch=3)
    try:
        xs = [np.random.default_rng(i).standard_normal((40, 50)).astype(np.float32) for i in range(7)]
        outs = [np.empty(1 << 16, np.uint8) for _ in xs]
        tickets = [srv.submit_compress(x, o, eb_rel=1e-3) for x, o in zip(xs, outs)]
        assert len(set(tickets)) == len(tickets)
        for t in tickets:
            st, n = srv.wait(t)
            assert st == szgb.ECUDA
        assert srv.stats()["completed"] == len(xs)
        with pytest.raises(szgb.SzgbError):
            srv.poll(tickets[0])  # released after completion
    finally:
        srv.close()


def test_server_request_log(szgb, tmp_path):
    import json
    log = tmp_path / "requests.jsonl"
    srv = szgb.Server(0, budget=64 << 20, workers=1, max_batch=2, log_path=str(log))
    try:
        xs = [np.random.default_rng(i).standard_normal((30, 20)).astype(np.float32) for i in range(3)]
        outs = [np.empty(1 << 16, np.uint8) for _ in xs]
        tickets = [srv.submit_compress(x, o, eb_rel=1e-3) for x, o in zip(xs, outs)]
        done = [srv.wait(t) for t in tickets[:2]]
        while not srv.poll(tickets[2])[0]:
            pass
    finally:
        srv.close()
    recs = [json.loads(line) for line in log.read_text().splitlines()]
    assert sorted(r["ticket"] for r in recs) == sorted(tickets)
    for r in recs:
        assert r["op"] == "compress" and r["shape"] == [30, 20] and r["in_bytes"] == 30 * 20 * 4
        assert r["latency_s"] >= 0.0
        if r["status"] == szgb.OK:  # with a GPU: the stream's own figures
            assert r["compression_factor"] == pytest.approx(r["in_bytes"] / r["out_bytes"])
        else:
            assert r["status"] == szgb.ECUDA and "compression_factor" not in r
    assert all(st in (szgb.OK, szgb.ECUDA) for st, _ in done)


def test_server_takes_every_field_kind(szgb, szo):
    # 3D fields with n = 3, 4, 4D fields and the lattice variant run alone on
    # their own kernels; the server admits them (compress, and decompress of
    # a 4D stream) like the fields the batched wavefront carries
    srv = szgb.Server(0, budget=64 << 20, workers=1, max_batch=2)
    try:
        x3 = np.zeros((6, 8, 10), np.float32)
        x4 = np.random.default_rng(5).standard_normal((2, 3, 8, 10)).astype(np.float32)
        tickets = []
        for x, kw in ((x3, dict(layers=3)), (x3, dict(layers=4)),
                      (x3, dict(layers=1, variant=szgb.VARIANT_LATTICE)), (x4, dict(layers=2))):
            tickets.append(srv.submit_compress(x, np.empty(1 << 16, np.uint8), eb_rel=1e-3, **kw))
        s4 = szo.compress(x4, eb_rel=1e-3, m=8)
        tickets.append(srv.submit_decompress(s4, np.empty(x4.shape, np.float32)))
        done = [srv.wait(t) for t in tickets]
        assert all(st in (szgb.OK, szgb.ECUDA) for st, _ in done)
        with pytest.raises(szgb.SzgbError) as e:  # too small for the 4D field
            srv.submit_decompress(s4, np.empty(x4.size - 1, np.float32))
        assert e.value.code == szgb.EINVAL
    finally:
        srv.close()
