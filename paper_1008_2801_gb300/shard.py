"""Sharding of independent solves across GPUs (one process per GPU).

The boxes of a batch (the grids of one MultiFAB level, paper Sec. 2, whose
FABs are distributed to nodes independently) and the right-hand sides of a
multi-RHS solve are independent problems: each rank solves its own share and
no data moves between ranks during the solve.  Shares are balanced by cell
count with the longest-processing-time rule (largest box first, to the least
loaded rank; ties to the lower rank), which is deterministic and within 4/3
of the optimal maximum load.
"""
from __future__ import annotations


def partition(cells, world: int):
    """Lists of box indices per rank for boxes of the given cell counts."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(cells)), key=lambda i: (-int(cells[i]), i))
    load = [0] * world
    out = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        out[r].append(i)
        load[r] += int(cells[i])
    return [sorted(o) for o in out]


def my_share(cells, rank: int, world: int):
    return partition(cells, world)[rank]
