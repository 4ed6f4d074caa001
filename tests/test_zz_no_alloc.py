"""gp_count_noalloc: the count for callers that cannot allocate device
memory (an arena owns it, the host application forbids cudaMalloc/cudaFree,
or the allocation latency is unacceptable). It must give exactly the
counts gp_count gives, call after call, since every call reuses the same
fixed device array. This file is collected last so that a failure here
comes after every other test has run."""

import numpy as np
import pytest

from synth import named_pattern, workload_edges

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def N():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2009_10955_gb300 import native
    return native()


def test_noalloc_matches_gp_count_on_consecutive_calls(N):
    graphs = {}
    for name in ("er2000", "rmat10"):
        n, s, d = workload_edges(name)
        graphs[name] = N.gp_graph_create_edges(s, d, n, N.GP_DEGREE_ORDER)
    calls = [("er2000", "house"), ("rmat10", "k4"), ("rmat10", "house"), ("er2000", "triangle")]
    for gname, pname in calls:
        g = graphs[gname]
        sch = N.gp_schedule(N.gp_pattern_create(named_pattern(pname)), g, top_k=1)
        expect = N.gp_count(g, sch, 0)
        assert expect[0] == N.GP_OK
        first = N.gp_count_noalloc(g, sch, 0)
        second = N.gp_count_noalloc(g, sch, 0)          # the array still holds the last call
        assert first == second == expect[1], (gname, pname)


def test_noalloc_rejects_plans_beyond_the_fixed_scratch(N):
    # a star with 4M leaves: the house plan keeps intermediate sets sized by
    # the maximum degree for every warp, far more than the fixed array holds
    # for even one block, so the call is refused before any launch
    leaves = 4_000_000
    src = np.zeros(leaves, dtype=np.int32)
    dst = np.arange(1, leaves + 1, dtype=np.int32)
    g = N.gp_graph_create_edges(src, dst, leaves + 1, N.GP_DEGREE_ORDER)
    sch = N.gp_schedule(N.gp_pattern_create(named_pattern("house")), g, top_k=1)
    with pytest.raises(N.GraphPiError) as e:
        N.gp_count_noalloc(g, sch, 0)
    assert e.value.status == N.GP_ERR_SCRATCH
    assert "fixed scratch" in str(e.value)
    # a refused call leaves the shared array usable
    n, s, d = workload_edges("er2000")
    small = N.gp_graph_create_edges(s, d, n, N.GP_DEGREE_ORDER)
    sch2 = N.gp_schedule(N.gp_pattern_create(named_pattern("house")), small, top_k=1)
    assert N.gp_count_noalloc(small, sch2, 0) == N.gp_count(small, sch2, 0)[1]
