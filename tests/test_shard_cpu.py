"""Multi-process (gloo, world size 2, CPU) checks of the host logic that
shards independent boxes across ranks and of the benchmark's rank helpers."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1008_2801_gb300 import inputs, shard


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, cells, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = shard.my_share(cells, rank, world)
        lists = [None] * world
        dist.all_gather_object(lists, mine)
        import bench
        mx = bench.max_over_ranks(float(rank + 1), torch.device("cpu"))
        bench.barrier()
        if rank == 0:
            q.put((lists, mx))
    finally:
        dist.destroy_process_group()


def test_two_ranks_cover_every_box_once():
    d = inputs.batched(64, 4)
    cells = [int(np.prod(x)) for x in d["dims"]]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, cells, q)) for r in range(2)]
    for p in procs:
        p.start()
    lists, mx = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert mx == 2.0
    flat = sorted(i for l in lists for i in l)
    assert flat == list(range(64))
    loads = [sum(cells[i] for i in l) for l in lists]
    lower = max(sum(cells) / 2, max(cells))
    assert max(loads) <= 4 / 3 * lower


@pytest.mark.parametrize("world", [1, 3, 8])
def test_partition_is_deterministic_and_balanced(world):
    r = np.random.default_rng(0)
    cells = list(r.integers(1, 10 ** 6, 50))
    a = shard.partition(cells, world)
    assert a == shard.partition(cells, world)
    assert sorted(i for l in a for i in l) == list(range(50))
    loads = [sum(cells[i] for i in l) for l in a]
    assert max(loads) <= 4 / 3 * max(sum(cells) / world, max(cells))
