"""The multi-GPU path's host logic on CPU: world-size-2 and -3 gloo ranks
shard the roots and sum partial counts exactly (the sharded path's one
exchange).
Partial counts come from the oracle's restricted enumeration per root range,
so the test needs no GPU."""

import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import oracle
from oracle import planner_ref as pr
from synth import er_edges, named_pattern


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    n = 120
    s, d = er_edges(n, 900, seed=21)
    g = oracle.build_csr(n, s, d)
    lo, hi = bench.shard_roots(g.row_ptr, rank, world)   # roots of this rank
    parts = []
    for name in ("triangle", "house", "c4"):
        adj = named_pattern(name)
        sched, _ = pr.efficient_schedules(adj.tolist())
        rs = pr.restriction_sets(adj.tolist())[0]
        parts.append(oracle.count_restricted(adj, sched[0], rs, g, root_begin=lo, root_end=hi, threads=1))
    # a value above 2^32 exercises the carry between halves
    parts.append((1 << 33) + rank * ((1 << 32) - 1))
    total = bench.allreduce_counts(parts)
    q.put((rank, total))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_ranks_shard_and_sum_exactly(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    n = 120
    s, d = er_edges(n, 900, seed=21)
    g = oracle.build_csr(n, s, d)
    expect = [oracle.count(named_pattern(x), g) for x in ("triangle", "house", "c4")]
    expect.append(world * (1 << 33) + (world * (world - 1) // 2) * ((1 << 32) - 1))
    assert all(res[r] == expect for r in range(world))


def test_shard_ranges_partition():
    import bench
    for ntasks in (0, 1, 7, 1000, 31400728):
        for world in (1, 2, 3, 8):
            rs = [bench.shard_range(ntasks, r, world) for r in range(world)]
            assert rs[0][0] == 0 and rs[-1][1] == ntasks
            assert all(a[1] == b[0] for a, b in zip(rs, rs[1:]))


def test_weighted_root_shards():
    """Root shards partition the roots and balance the sum of squared
    degrees to within one root."""
    import bench
    from synth import workload_edges
    n, s, d = workload_edges("rmat12")
    g = oracle.build_csr(n, s, d)
    deg = np.diff(g.row_ptr).astype(np.float64)
    w = deg * deg
    for world in (1, 2, 3, 8):
        rs = [bench.shard_roots(g.row_ptr, r, world) for r in range(world)]
        assert rs[0][0] == 0 and rs[-1][1] == n
        assert all(a[1] == b[0] and a[0] <= a[1] for a, b in zip(rs, rs[1:]))
        for lo, hi in rs:
            assert w[lo:hi].sum() <= w.sum() / world + w.max()
    assert bench.shard_roots(np.zeros(1, np.int64), 0, 2) == (0, 0)


class _FakeSchedules:
    """A plan as the sharding layer sees it: its divisor via iep()."""

    def __init__(self, adj, div):
        self.adj = adj
        self.order = tuple(pr.efficient_schedules(adj.tolist())[0][0])
        self.res = pr.restriction_sets(adj.tolist())[0]
        self.div = div

    def iep(self, idx):
        return (2 if self.div > 1 else 0), self.div


class _FakeNative:
    """Stands in for the library's count call: the undivided total of an
    edge-task range is the oracle's count over those CSR entries times the
    plan's divisor, so the layer's partition, reduction and division are
    what is tested."""
    GP_OK = 0

    def __init__(self, g):
        self.g = g

    def gp_count_raw(self, graph, sched, idx, stream=None, task_begin=0, task_end=0):
        c = oracle.count_restricted_entries(sched.adj, sched.order, sched.res, self.g, task_begin, task_end,
                                            threads=1)
        return self.GP_OK, c * sched.div


def _sharded_main(rank, world, port, q):
    import torch.distributed as dist
    from paper_2009_10955_gb300 import shard
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    n = 150
    s, d = er_edges(n, 1100, seed=23)
    g = oracle.build_csr(n, s, d)
    shard.N = _FakeNative(g)
    shard.graph_row_ptr = lambda graph: g.row_ptr
    out = [shard.count_sharded(None, _FakeSchedules(named_pattern(x), div), 0)
           for x, div in (("triangle", 1), ("house", 1), ("house", 2), ("diamond", 6))]
    q.put((rank, out))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_count_sharded_over_gloo_ranks(world):
    """paper_2009_10955_gb300.shard.count_sharded: every rank counts the
    edge tasks of its roots, one all-reduce sums the undivided totals and the
    divisor applies after the sum; every rank returns the whole count."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_sharded_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    n = 150
    s, d = er_edges(n, 1100, seed=23)
    g = oracle.build_csr(n, s, d)
    expect = [oracle.count(named_pattern(x), g) for x in ("triangle", "house", "house", "diamond")]
    assert all(res[r] == expect for r in range(world))


def test_rank_tasks_and_finish_count():
    from paper_2009_10955_gb300 import shard
    n, s, d = 200, *er_edges(200, 1500, seed=4)
    g = oracle.build_csr(n, s, d)
    for world in (1, 2, 5):
        rs = [shard.rank_tasks(g.row_ptr, r, world) for r in range(world)]
        assert rs[0][0] == 0 and rs[-1][1] == int(g.row_ptr[-1])
        assert all(a[1] == b[0] for a, b in zip(rs, rs[1:]))
    assert shard.finish_count(12, 3) == 4
    with pytest.raises(ArithmeticError):
        shard.finish_count(13, 3)
    with pytest.raises(OverflowError):
        shard.finish_count(1 << 70, 1)
