"""Assignment of independent fields to GPUs (one process per GPU).

Fields are independent units of the method: each is compressed on its own,
with no exchange between fields, which is how the paper runs in parallel
(one process per field or group of fields, no communication).  A single field
is never split, because cutting it would change the predictions at the cut
and therefore the stream.  Fields go to ranks greedily, largest first, each
to the rank with the fewest bytes so far (ties to the lowest rank): every
rank computes the same assignment from the same sizes, so no collective is
needed on the data path.
"""
from __future__ import annotations


def assign_fields(nbytes, world: int):
    """List, per rank, of the indices of the fields it owns (ascending)."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(nbytes)), key=lambda i: (-int(nbytes[i]), i))
    load = [0] * world
    owned = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        owned[r].append(i)
        load[r] += int(nbytes[i])
    return [sorted(o) for o in owned]


def my_fields(nbytes, world: int, rank: int):
    return assign_fields(nbytes, world)[rank]
