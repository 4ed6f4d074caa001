"""gp_count_noalloc: the count for callers that cannot allocate device
memory while they count (an arena or pool owns all of it, the host
application forbids cudaMalloc/cudaFree on its streams, or an allocation's
latency is unacceptable). It must give exactly the counts gp_count and the
oracle give, call after call, since every call reuses the same fixed device
array, and it must allocate nothing: the device's memory pool (where
gp_count's stream-ordered allocations come from) sees no new use. This file
is collected last so that a failure here comes after every other test has
run."""

import ctypes
import os

import numpy as np
import pytest

import oracle
from synth import named_pattern, workload_edges

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def N():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2009_10955_gb300 import native
    return native()


def _cudart():
    for name in ("/usr/local/cuda/lib64/libcudart.so", "libcudart.so.13", "libcudart.so"):
        try:
            return ctypes.CDLL(name)
        except OSError:
            continue
    pytest.skip("libcudart not found")


class Pool:
    """The current memory pool of device 0, as cudaMallocAsync uses it."""
    USED_CURRENT, USED_HIGH, RESERVED_CURRENT = 7, 8, 5      # cudaMemPoolAttr values

    def __init__(self):
        self.rt = _cudart()
        self.h = ctypes.c_void_p()
        assert self.rt.cudaDeviceGetMemPool(ctypes.byref(self.h), 0) == 0

    def get(self, attr):
        v = ctypes.c_uint64()
        assert self.rt.cudaMemPoolGetAttribute(self.h, attr, ctypes.byref(v)) == 0
        return v.value

    def reset_high(self):
        zero = ctypes.c_uint64(0)
        assert self.rt.cudaMemPoolSetAttribute(self.h, self.USED_HIGH, ctypes.byref(zero)) == 0


def oracle_pair(n, s, d):
    ref, _ = oracle.degree_relabel(oracle.build_csr(n, s, d))
    return ref


def test_noalloc_matches_gp_count_on_consecutive_calls(N):
    graphs = {}
    for name in ("er2000", "rmat10"):
        n, s, d = workload_edges(name)
        graphs[name] = (N.gp_graph_create_edges(s, d, n, N.GP_DEGREE_ORDER), oracle_pair(n, s, d))
    calls = [("er2000", "house"), ("rmat10", "k4"), ("rmat10", "house"), ("er2000", "triangle")]
    for gname, pname in calls:
        g, ref = graphs[gname]
        sch = N.gp_schedule(N.gp_pattern_create(named_pattern(pname)), g, top_k=1)
        expect = N.gp_count(g, sch, 0)
        assert expect[0] == N.GP_OK
        first = N.gp_count_noalloc(g, sch, 0)
        second = N.gp_count_noalloc(g, sch, 0)          # the array still holds the last call
        assert first == second == expect[1], (gname, pname)
        assert first == oracle.count(named_pattern(pname), ref), (gname, pname)


def test_noalloc_allocates_nothing(N):
    import torch
    n, s, d = workload_edges("rmat10")
    g = N.gp_graph_create_edges(s, d, n, N.GP_DEGREE_ORDER)
    sch = N.gp_schedule(N.gp_pattern_create(named_pattern("house")), g, top_k=1)
    expect = N.gp_count_noalloc(g, sch, 0)              # warm: the array is in place
    torch.cuda.synchronize()
    pool = Pool()
    used0, reserved0 = pool.get(Pool.USED_CURRENT), pool.get(Pool.RESERVED_CURRENT)
    pool.reset_high()
    assert N.gp_count_noalloc(g, sch, 0) == expect
    torch.cuda.synchronize()
    assert pool.get(Pool.USED_HIGH) <= used0
    assert pool.get(Pool.RESERVED_CURRENT) == reserved0
    # the check is sensitive: gp_count allocates its scratch from this pool
    pool.reset_high()
    assert N.gp_count(g, sch, 0)[1] == expect
    torch.cuda.synchronize()
    assert pool.get(Pool.USED_HIGH) > used0


def test_noalloc_with_a_grid_shrunk_to_the_array(N):
    """A hub of 200,000 neighbours: the intermediate sets of one block of 8
    warps take several MB, so only a few blocks fit in the fixed array and the
    launch runs on a grid far below the SM count; counts still equal
    gp_count and the oracle's restricted enumeration with the same plan."""
    n, hub = 250_000, 200_000
    rng = np.random.default_rng(17)
    s = np.concatenate([np.zeros(hub, np.int32), rng.integers(0, n, 600_000).astype(np.int32)])
    d = np.concatenate([np.arange(1, hub + 1, dtype=np.int32), rng.integers(0, n, 600_000).astype(np.int32)])
    g = N.gp_graph_create_edges(s, d, n, N.GP_DEGREE_ORDER)
    assert g.stats(with_triangles=False)["max_deg"] >= hub
    ref = oracle_pair(n, s, d)
    # plans whose first vertex is the largest id of the first two: the hub
    # (id 0 in the degree order) is never a root, so the oracle's walk stays
    # short, while the kernel's sets still need the hub's 200,000 entries
    plans = {"triangle": ((0, 1, 2), [(0, 1), (1, 2)]),
             "k4": ((0, 1, 2, 3), [(0, 1), (1, 2), (2, 3)]),
             "diamond": ((0, 1, 2, 3), [(0, 1), (2, 3)])}
    for pname, (order, res) in plans.items():
        adj = named_pattern(pname)
        sch = N.gp_schedule_explicit(N.gp_pattern_create(adj), order, res)
        got = N.gp_count_noalloc(g, sch, 0)
        assert got == N.gp_count(g, sch, 0)[1] == oracle.count_restricted(adj, order, res, ref), pname
        assert N.gp_count_noalloc(g, sch, 0) == got


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
