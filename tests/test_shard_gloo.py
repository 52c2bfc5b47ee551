"""Field sharding across ranks, checked with world_size 2 over gloo on CPU:
every field is owned by exactly one rank, the ranks agree without exchanging
data, the byte load is balanced within one field's size, and the streams each
rank produces for its own fields (with the oracle; the GPU path's streams are
the oracle's bytes) equal the single-process streams."""
import os

import pytest

from paper_1706_03791_gb300.shard import assign_fields


def test_assignment_properties():
    sizes = [100, 3, 50, 50, 7, 90, 1, 64, 64, 2]
    for world in (1, 2, 3, 4, 16):
        owned = assign_fields(sizes, world)
        flat = sorted(i for o in owned for i in o)
        assert flat == list(range(len(sizes)))
        loads = [sum(sizes[i] for i in o) for o in owned]
        assert max(loads) - min(loads) <= max(sizes)
    with pytest.raises(ValueError):
        assign_fields(sizes, 0)


def _worker(rank, world, port, sizes, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_1706_03791_gb300.shard import my_fields
    mine = my_fields(sizes, world, rank)
    got = [None] * world
    dist.all_gather_object(got, mine)
    load = sum(sizes[i] for i in mine)
    import torch
    t = torch.tensor([load], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)  # the job's time is the slowest rank's
    if rank == 0:
        q.put((got, float(t.item())))
    dist.barrier()
    dist.destroy_process_group()


def test_gloo_world2():
    import socket
    import torch.multiprocessing as mp
    sizes = [int(s) for s in (1800 * 3600 * 4, 64 ** 3 * 4, 2048 ** 2 * 4, 256 ** 3 * 4, 100, 7, 512 * 512 * 4)]
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, sizes, q)) for r in range(2)]
    for p in procs:
        p.start()
    got, maxload = q.get(timeout=120)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    flat = sorted(i for o in got for i in o)
    assert flat == list(range(len(sizes)))
    assert set(got[0]).isdisjoint(got[1])
    assert maxload == max(sum(sizes[i] for i in o) for o in got)


def _small_uneven(i):
    """Field i of a small uneven batch (2D and 3D k^-3 fields of mixed size)."""
    import numpy as np
    from synthetic import fields
    rng = np.random.default_rng(700 + i)
    if i % 2 == 0:
        n0, n1 = int(rng.integers(20, 90)), int(rng.integers(20, 120))
        x = fields.grf2d(n0, n1, seed=800 + i)
    else:
        s = [int(v) for v in rng.integers(5, 24, 3)]
        x = fields.blobs3d(*s, seed=800 + i, nblobs=3)
    eb = (1e-3, 1e-4, 1e-5)[i % 3]
    return x, eb


def _data_worker(rank, world, port, nfields, q):
    """Each rank compresses the fields it owns with the oracle; rank 0
    gathers (field index, stream) from every rank."""
    import hashlib
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from oracle import szo
    from paper_1706_03791_gb300.shard import my_fields
    sizes = [_small_uneven(i)[0].nbytes for i in range(nfields)]
    out = {}
    for i in my_fields(sizes, world, rank):
        x, eb = _small_uneven(i)
        s = szo.compress(x, eb_rel=eb, m=0)
        out[i] = (hashlib.sha256(bytes(s)).hexdigest(), int(s.size))
    got = [None] * world
    dist.all_gather_object(got, out)  # host-side gather of (field, stream) only
    if rank == 0:
        q.put(got)
    dist.barrier()
    dist.destroy_process_group()


def test_gloo_world2_streams_match_single_process(szo):
    """Sharding is rank-independent: the streams two ranks produce for their
    own fields are exactly the single-process streams of those fields."""
    import hashlib
    import socket
    import torch.multiprocessing as mp
    nfields = 12
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_data_worker, args=(r, 2, port, nfields, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = q.get(timeout=180)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert set(got[0]).isdisjoint(got[1]) and set(got[0]) | set(got[1]) == set(range(nfields))
    assert got[0] and got[1]  # both ranks did work
    merged = {**got[0], **got[1]}
    for i in range(nfields):
        x, eb = _small_uneven(i)
        s = szo.compress(x, eb_rel=eb, m=0)
        assert merged[i] == (hashlib.sha256(bytes(s)).hexdigest(), int(s.size)), i
