"""One process per GPU: independent LPs are sharded over the ranks with no
data-path collective (the successive-fixing rounds of many instances and
the batch family are independent relaxations; one LP solve does not
shard, so a single-LP job runs one replica per rank).  Host logic only; the
collectives here (timing, gathering results) carry scalars and small
Python objects."""
from __future__ import annotations


def shard(sizes, rank: int, world: int) -> list:
    """Indices of the items rank ``rank`` solves: longest-processing-time
    assignment by size (largest first, to the least-loaded rank, ties to the
    lowest rank), so every rank gets a near-equal share of nonzeros.  The
    shards are disjoint, cover every item and do not depend on the rank
    that computes them."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank %d out of range for world size %d" % (rank, world))
    order = sorted(range(len(sizes)), key=lambda i: (-sizes[i], i))
    load = [0] * world
    mine = []
    for i in order:
        r = min(range(world), key=lambda q: (load[q], q))
        load[r] += sizes[i]
        if r == rank:
            mine.append(i)
    return sorted(mine)


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """The largest value over the ranks (the job's time is its slowest
    rank's); the value itself without a process group."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def gather_on_rank0(obj, dist=None):
    """Every rank's object, in rank order, on rank 0 (None elsewhere)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return [obj]
    out = [None] * dist.get_world_size() if dist.get_rank() == 0 else None
    dist.gather_object(obj, out, dst=0)
    return out
