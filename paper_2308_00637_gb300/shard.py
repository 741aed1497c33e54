"""Multi-GPU sharding of a batch of independent QPs (one process per GPU).

The QPs of a batch share nothing, so the batch is split across ranks with no
collective on the data path: each rank solves its shard with the batched
solver on its own GPU, and the solutions are gathered once at the end.  The
split is longest-processing-time-first (LPT) on the work of one K*v product,
which for a dense QP is proportional to n^2 + m*n (the bytes of H and A).

``lpt_shards`` is pure host logic; ``solve_sharded`` takes the per-rank solve
as a callable so that the partition and the gather can be tested with gloo
ranks on CPU.
"""
from __future__ import annotations

from typing import Callable, List, Sequence


def qp_cost(n: int, m: int) -> float:
    """Work of one K*v product of a dense QP: the entries of H and A."""
    return float(n) * n + float(m) * n


def lpt_shards(costs: Sequence[float], world: int) -> List[List[int]]:
    """Indices of the QPs each rank solves: largest cost first, each onto the
    currently least-loaded rank (ties to the lower rank).  Every index appears
    in exactly one shard; each shard is in ascending index order."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    load = [0.0] * world
    shards: List[List[int]] = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        shards[r].append(i)
        load[r] += costs[i]
    return [sorted(s) for s in shards]


def solve_sharded(qps: Sequence, solve_shard: Callable, rank: int, world: int, dist=None):
    """Solve `qps` across `world` ranks.  `solve_shard(list_of_qps)` returns
    one result per QP (any picklable object, e.g. the solution vector); the
    results of all ranks are gathered (one all_gather_object at the end, no
    collective during the solves) and returned in the order of `qps` on
    every rank."""
    shards = lpt_shards([qp_cost(q.n, q.m) for q in qps], world)
    mine = shards[rank]
    res = solve_shard([qps[i] for i in mine]) if mine else []
    if len(res) != len(mine):
        raise RuntimeError("solve_shard returned a wrong number of results")
    if world == 1 or dist is None:
        parts = [list(zip(mine, res))]
    else:
        parts = [None] * world
        dist.all_gather_object(parts, list(zip(mine, res)))
    out = [None] * len(qps)
    for part in parts:
        for i, r in part:
            if out[i] is not None:
                raise RuntimeError(f"QP {i} solved twice")
            out[i] = r
    if any(o is None for o in out):
        raise RuntimeError("a QP was not solved")
    return out


def batch_solve_fn(opts=None):
    """The per-rank solve for `solve_sharded`: the batched GPU solver
    (qp_create_batch + ipm_solve_batch) on the rank's current device;
    returns, per QP, (status, x)."""
    import numpy as np
    from . import qp_create_batch, ipm_solve_batch, qp_batch_destroy

    def run(shard):
        b = qp_create_batch(shard)
        xs = [np.zeros(q.n) for q in shard]
        _, status, _ = ipm_solve_batch(b, opts, xs)
        qp_batch_destroy(b)
        return list(zip(status, xs))
    return run
