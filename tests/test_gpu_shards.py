"""The sharded path of the benchmark on one GPU: every rank's share of the
edge tasks (whole roots, balanced by the sum of squared degrees) is counted
as that rank would count it, and the undivided totals of the shares add up
to the whole count, for plain and inclusion-exclusion plans. The ranks'
launches are independent (no rank waits on another), so running them one
after another on one GPU is the same computation."""

import pytest

import bench
from synth import named_pattern, workload_edges

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2009_10955_gb300 import native
    N = native()
    n, s, d = workload_edges("rmat14")
    return N, N.gp_graph_create_edges(s, d, n, N.GP_DEGREE_ORDER)


@pytest.mark.parametrize("pname,iep", [("triangle", False), ("k4", False), ("house", True), ("star5", True),
                                       ("k5", False)])
@pytest.mark.parametrize("world", [2, 3, 8])
def test_shards_add_up(env, pname, iep, world):
    N, g = env
    sc = N.gp_schedule(N.gp_pattern_create(named_pattern(pname)), g)
    if iep:
        assert sc.set_iep(True) == 1
    whole = N.gp_count(g, sc)[1]
    rp = g.csr()[0]
    total = 0
    for rank in range(world):
        r0, r1 = bench.shard_roots(rp, rank, world)
        if rp[r0] == rp[r1]:
            continue                            # an empty share (task_end 0 would mean all tasks)
        st, raw = N.gp_count_raw(g, sc, 0, task_begin=int(rp[r0]), task_end=int(rp[r1]) if r1 < len(rp) - 1 else 0)
        assert st == N.GP_OK
        total += raw
    div = sc.iep(0)[1]
    assert total % div == 0 and total // div == whole


@pytest.mark.parametrize("pname,iep", [("k4", False), ("house", True)])
def test_package_rank_totals_add_up(env, pname, iep):
    """The package's sharding layer (shard.rank_total over shard.graph_row_ptr,
    as count_sharded runs it on each rank) on one GPU, rank after rank."""
    from paper_2009_10955_gb300 import shard
    N, g = env
    sc = N.gp_schedule(N.gp_pattern_create(named_pattern(pname)), g)
    if iep:
        assert sc.set_iep(True) == 1
    whole = N.gp_count(g, sc)[1]
    rp = shard.graph_row_ptr(g)
    assert (rp == g.csr()[0]).all()
    for world in (1, 3):
        total = sum(shard.rank_total(g, sc, 0, rank, world, row_ptr=rp) for rank in range(world))
        assert shard.finish_count(total, sc.iep(0)[1]) == whole
    assert shard.count_sharded(g, sc) == whole          # one process: every task on this rank
