"""Field sharding across ranks, checked with world_size 2 over gloo on CPU:
every field is owned by exactly one rank, the ranks agree without exchanging
data, and the byte load is balanced within one field's size."""
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
