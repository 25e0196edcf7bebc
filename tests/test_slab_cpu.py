"""Host logic of the slab-decomposed box (no GPU): the slab plan and the halo
bookkeeping of mg_slab_plan / mg_slab_halo, checked on their own and by two
gloo ranks that each hold one slab, exchange their boundary planes with the
library's halo records and apply a 7-point stencil locally: the result must
be the stencil of the whole box."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1008_2801_gb300 import MGError, slab_halo, slab_plan


def test_plan_splits_equal_slabs_and_gathers_at_32_cubed():
    z0, g = slab_plan((512, 512, 512), 2)
    assert z0 == [0, 256, 512]
    assert g == 4            # 512 -> 256 -> 128 -> 64 -> 32: 32^3 cells are gathered
    z0, g = slab_plan((512, 512, 512), 8)
    assert z0 == list(range(0, 513, 64)) and g == 4
    z0, g = slab_plan((64, 48, 40), 2)   # (nz, ny, nx)
    assert z0 == [0, 32, 64] and g == 1  # 40 x 48 x 64 -> 20 x 24 x 32 <= 32^3
    # a slab of 4 planes halves twice; the level where it is 1 plane thick stops
    z0, g = slab_plan((16, 256, 256), 4)
    assert g == 2


@pytest.mark.parametrize("shape,nslab", [((63, 64, 64), 2), ((64, 64, 64), 3),
                                         ((32, 32, 32), 2), ((64, 64, 65), 2)])
def test_plan_rejects_what_does_not_split(shape, nslab):
    with pytest.raises(MGError) as ei:
        slab_plan(shape, nslab)
    assert ei.value.name in ("unsupported", "invalid_arg")


def test_halo_records_pair_every_interface():
    shape, nslab = (256, 64, 64), 4
    z0, g = slab_plan(shape, nslab)
    for level in range(g):
        t = (z0[1] - z0[0]) >> level
        recs = slab_halo(shape, nslab, level)
        assert len(recs) == 2 * (nslab - 1)
        for r in range(nslab - 1):
            assert {"src": r, "src_k": t - 1, "dst": r + 1, "dst_k": -1} in recs
            assert {"src": r + 1, "src_k": 0, "dst": r, "dst_k": t} in recs
    with pytest.raises(MGError):
        slab_halo(shape, nslab, g)


def _laplacian(u):
    """7-point stencil with zero values outside the array (no scaling)."""
    p = np.pad(u, 1)
    return (p[:-2, 1:-1, 1:-1] + p[2:, 1:-1, 1:-1] + p[1:-1, :-2, 1:-1] + p[1:-1, 2:, 1:-1] +
            p[1:-1, 1:-1, :-2] + p[1:-1, 1:-1, 2:] - 6 * u)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, shape, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        z0, g = slab_plan(shape, world)
        glob = np.random.default_rng(7).standard_normal(shape)
        out = []
        for level in range(g):
            # the level's field: every rank draws the same global array and
            # keeps its slab in a local array with one guard plane each side
            f = 2 ** level
            u = glob[::f, ::f, ::f] if level else glob
            t = (z0[1] - z0[0]) >> level
            mine = u[rank * t:(rank + 1) * t]
            loc = np.zeros((t + 2,) + u.shape[1:])
            loc[1:-1] = mine
            reqs = []
            for h in slab_halo(shape, world, level):
                if h["src"] == rank:
                    buf = torch.from_numpy(np.ascontiguousarray(loc[h["src_k"] + 1]))
                    reqs.append(dist.isend(buf, dst=h["dst"]))
            for h in slab_halo(shape, world, level):
                if h["dst"] == rank:
                    buf = torch.empty(u.shape[1:], dtype=torch.float64)
                    dist.recv(buf, src=h["src"])
                    loc[h["dst_k"] + 1] = buf.numpy()
            for rq in reqs:
                rq.wait()
            # the stencil of the slab's cells from the local array (guards
            # hold the neighbours' planes, or 0 at the box's walls)
            p = np.pad(loc, ((0, 0), (1, 1), (1, 1)))
            c = p[1:-1, 1:-1, 1:-1]
            lap = (p[:-2, 1:-1, 1:-1] + p[2:, 1:-1, 1:-1] + p[1:-1, :-2, 1:-1] +
                   p[1:-1, 2:, 1:-1] + p[1:-1, 1:-1, :-2] + p[1:-1, 1:-1, 2:] - 6 * c)
            want = _laplacian(u)[rank * t:(rank + 1) * t]
            out.append(float(np.max(np.abs(lap - want))))
        q.put((rank, out))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_exchange_halos_by_the_library_records():
    shape = (128, 64, 48)    # (nz, ny, nx): two slab levels, gathered at level 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, shape, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert len(res[0]) >= 2
    for r in (0, 1):
        assert max(res[r]) == 0.0, res
