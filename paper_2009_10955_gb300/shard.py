"""One count sharded over ranks, one process per GPU (Section IV-E: the
graph is replicated, the edge tasks are independent).

Every rank holds a replica of the graph and counts the edge tasks of a
contiguous range of root vertices; the ranges are cut so that they carry
about the same estimated work (a root of degree d owns d edge tasks of
about d steps each, so a range weighs the sum of its roots' d^2). The one
exchange is the exact sum of the ranks' undivided 128-bit totals; an
inclusion-exclusion plan's total is divided by its divisor only after the
sum (Section IV-D), so such plans shard too.

The partition and the reduction are host logic; every count runs in the
library's kernels.
"""

import numpy as np

from . import _native as N


def shard_range(ntasks, rank, world):
    """Contiguous share [lo, hi) of ntasks edge tasks for one rank."""
    return ntasks * rank // world, ntasks * (rank + 1) // world


def shard_roots(row_ptr, rank, world):
    """Contiguous root range [lo, hi) of one rank, cut by the cumulative sum
    of squared degrees. The ranges partition the roots; a rank's weight
    exceeds the mean by at most one root's."""
    rp = np.asarray(row_ptr, dtype=np.int64)
    deg = np.diff(rp).astype(np.float64)
    cum = np.concatenate([[0.0], np.cumsum(deg * deg)])
    n = len(rp) - 1

    def cut(r):
        if r <= 0:
            return 0
        if r >= world:
            return n
        return min(n, int(np.searchsorted(cum, cum[-1] * r / world, side="left")))
    return cut(rank), cut(rank + 1)


def graph_row_ptr(graph):
    """The graph's CSR row offsets (n + 1 int64, host), without its lists."""
    n = graph.stats(with_triangles=False)["n"]
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    N.check(N.lib().gp_graph_copy_csr(graph.h, N._ptr(row_ptr), None, None), "gp_graph_copy_csr")
    return row_ptr


def rank_tasks(row_ptr, rank, world):
    """Edge-task range [lo, hi) (CSR entries) owned by one rank: the entries
    of its roots."""
    r0, r1 = shard_roots(row_ptr, rank, world)
    return int(row_ptr[r0]), int(row_ptr[r1])


def rank_total(graph, schedules, idx, rank, world, row_ptr=None, stream=None, **kw):
    """Undivided 128-bit total of one rank's edge tasks (0 for an empty
    share). Extra keywords go to make_opts (launch knobs)."""
    if row_ptr is None:
        row_ptr = graph_row_ptr(graph)
    lo, hi = rank_tasks(row_ptr, rank, world)
    if hi <= lo:                                   # task_end 0 would mean all tasks
        return 0
    status, raw = N.gp_count_raw(graph, schedules, idx, stream=stream, task_begin=lo, task_end=hi, **kw)
    if status != N.GP_OK:
        raise N.GraphPiError(status, f"rank {rank}: count returned status {status}")
    return raw


def allreduce_counts(counts, device=None):
    """Exact sum over the ranks of torch.distributed of non-negative integer
    totals (< 2^128 each and in total): each travels as four 32-bit limbs in
    int64 lanes, which cannot overflow for fewer than 2^31 ranks."""
    import torch
    import torch.distributed as dist
    limbs = torch.tensor([[(c >> (32 * i)) & 0xFFFFFFFF for i in range(4)] for c in counts],
                         dtype=torch.int64, device=device)
    dist.all_reduce(limbs)
    return [sum(int(x) << (32 * i) for i, x in enumerate(row)) for row in limbs.tolist()]


def finish_count(total, divisor):
    """The count from a summed undivided total: exact division by the plan's
    divisor, and the result must fit in 64 bits (the library's count width)."""
    if total % divisor:
        raise ArithmeticError(f"total {total} is not a multiple of the divisor {divisor}")
    count = total // divisor
    if count >> 64:
        raise OverflowError(f"count {count} needs more than 64 bits")
    return count


def count_sharded(graph, schedules, idx=0, stream=None, device=None, **kw):
    """The count of plan idx with this process's rank counting its share of
    the edge tasks and one all-reduce summing the shares (a single process
    counts everything). Every rank returns the same count."""
    import torch.distributed as dist
    world = dist.get_world_size() if dist.is_available() and dist.is_initialized() else 1
    rank = dist.get_rank() if world > 1 else 0
    total = rank_total(graph, schedules, idx, rank, world, stream=stream, **kw)
    if world > 1:
        total = allreduce_counts([total], device=device)[0]
    return finish_count(total, schedules.iep(idx)[1])
