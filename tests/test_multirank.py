"""Host logic of the N-replica benchmark path (one process per GPU): the
timing each rank reports is reduced to the slowest rank's, over a real
torch.distributed process group.  Run on the CPU with two `gloo` ranks."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t = bench.max_over_ranks(1.5 + rank, dist, "cpu")
    q.put((rank, t))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_gloo_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = dict(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert out == {0: 2.5, 1: 2.5}


def test_max_over_ranks_single_process():
    import bench
    assert bench.max_over_ranks(3.25, None, "cpu") == 3.25


# ---------------------------------------------------------------- batch sharding (LPT, no collective)
def test_lpt_shards_cover_and_balance():
    import qpgen
    from paper_2308_00637_gb300.shard import lpt_shards, qp_cost
    sizes = qpgen.batch_sizes(512, 64, 4096)
    costs = [qp_cost(n, n // 2) for n in sizes]
    for world in (1, 2, 3, 8):
        shards = lpt_shards(costs, world)
        flat = sorted(i for s in shards for i in s)
        assert flat == list(range(len(sizes)))
        loads = [sum(costs[i] for i in s) for s in shards]
        # LPT: the largest load is within one job of the average
        assert max(loads) <= sum(costs) / world + max(costs)
        assert all(s == sorted(s) for s in shards)


def _fake_solve(shard):
    """Stand-in for the per-rank GPU batch solve (CPU): a value that depends
    on the QP alone, so the gathered order can be checked."""
    import numpy as np
    return [(q.n, float(np.sum(q.p))) for q in shard]


def _shard_worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import qpgen
    from paper_2308_00637_gb300.shard import lpt_shards, qp_cost, solve_sharded
    sizes = qpgen.batch_sizes(24, 16, 200, size_seed=7)
    qps = [qpgen.batch_qp(k, n) for k, n in enumerate(sizes)]
    seen = []

    def solve(shard):
        seen.extend(qq.n for qq in shard)
        return _fake_solve(shard)
    out = solve_sharded(qps, solve, rank, world, dist)
    mine = lpt_shards([qp_cost(x.n, x.m) for x in qps], world)[rank]
    q.put((rank, out, seen, [qps[i].n for i in mine]))
    dist.barrier()
    dist.destroy_process_group()


def test_solve_sharded_gloo_two_ranks():
    import qpgen
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict((r, (o, s, m)) for r, o, s, m in (q.get(timeout=120) for _ in range(2)))
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    sizes = qpgen.batch_sizes(24, 16, 200, size_seed=7)
    ref = _fake_solve([qpgen.batch_qp(k, n) for k, n in enumerate(sizes)])
    for r in (0, 1):
        out, seen, mine = res[r]
        assert [tuple(x) for x in out] == ref          # every rank holds all results, in order
        assert seen == mine and len(seen) > 0           # each rank solved exactly its shard
    assert sorted(res[0][1] + res[1][1]) == sorted(sizes)
