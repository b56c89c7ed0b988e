"""Host logic of the multi-GPU path on CPU: two gloo ranks (127.0.0.1) shard
independent LPs (disjoint, covering, balanced by nonzeros), take the job
time as the slowest rank's, and gather their results on rank 0."""
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_2510_10891_b300.ranks import gather_on_rank0, max_over_ranks, shard


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, sizes, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = shard(sizes, rank, world)
        t = max_over_ranks(1.0 + rank, dist)
        got = gather_on_rank0({"rank": rank, "items": mine, "nnz": sum(sizes[i] for i in mine)}, dist)
        q.put((rank, mine, t, got))
    finally:
        dist.destroy_process_group()


def test_shard_single_process():
    sizes = [5, 3, 9, 1, 7, 7, 2]
    parts = [shard(sizes, r, 3) for r in range(3)]
    assert sorted(sum(parts, [])) == list(range(len(sizes)))
    loads = [sum(sizes[i] for i in p) for p in parts]
    assert max(loads) - min(loads) <= max(sizes)
    assert shard(sizes, 0, 1) == list(range(len(sizes)))
    with pytest.raises(ValueError):
        shard(sizes, 3, 3)
    assert max_over_ranks(2.5) == 2.5


def test_two_gloo_ranks():
    from scuc_gen import batch_configs
    sizes = [c.buses * c.T for c in batch_configs(64, 1000)]     # stand-in for each LP's nonzeros
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, sizes, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = {}
    for _ in range(world):
        rank, mine, t, got = q.get(timeout=120)
        res[rank] = (mine, t, got)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    a, b = res[0][0], res[1][0]
    assert not set(a) & set(b) and sorted(a + b) == list(range(len(sizes)))
    la, lb = sum(sizes[i] for i in a), sum(sizes[i] for i in b)
    assert abs(la - lb) <= max(sizes)
    assert res[0][1] == res[1][1] == 2.0                          # the slowest rank's time
    got = res[0][2]
    assert [g["rank"] for g in got] == [0, 1] and got[0]["items"] == a and got[1]["items"] == b
    assert res[1][2] is None
