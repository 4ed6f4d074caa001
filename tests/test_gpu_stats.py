"""The instrumented kernel (GP_COUNT_STATS) runs the same paths as the plain
one: it gives the same counts, tallies bitmap word operations exactly when
the bitmap subtree runs, and list bytes when lists are intersected."""

import ctypes

import pytest

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


def stats(N, g, sc, flags=0):
    b, o = ctypes.c_uint64(), ctypes.c_uint64()
    opts = N.make_opts(flags=N.GP_COUNT_STATS | flags, algo_bytes=ctypes.pointer(b), algo_ops=ctypes.pointer(o))
    st, c = N.gp_count(g, sc, 0, opts)
    return c, b.value, o.value


@pytest.mark.parametrize("pname", ["triangle", "k4", "k5", "house", "diamond"])
def test_instrumented_counts_and_tallies(env, pname):
    N, g = env
    sc = N.gp_schedule(N.gp_pattern_create(named_pattern(pname)), g)
    plain = N.gp_count(g, sc)[1]
    c, b, o = stats(N, g, sc)
    assert c == plain
    assert b > 0                               # every plan intersects some lists
    if pname in ("k4", "k5"):                  # clique plans run the bitmap subtree on core tasks
        assert o > 0
    if pname in ("triangle", "house"):         # no bitmap subtree for these plans
        assert o == 0
    c2, b2, o2 = stats(N, g, sc, N.GP_COUNT_NO_CORE)
    assert c2 == plain and o2 == 0 and b2 >= b


def test_busy_cycles(env):
    """Busy warp cycles: positive, the launched warps a multiple of 8 (whole
    blocks), and a count over half of the tasks is busy for less than the
    whole count (the same plan, the same grid)."""
    N, g = env
    sc = N.gp_schedule(N.gp_pattern_create(named_pattern("house")), g)
    nnz = g.device_csr()[2]

    def busy(**kw):
        b = (ctypes.c_uint64 * 2)()
        N.gp_count(g, sc, 0, N.make_opts(busy_cycles=ctypes.cast(b, ctypes.POINTER(ctypes.c_uint64)), **kw))
        return b[0], b[1]

    whole, warps = busy()
    assert whole > 0 and warps > 0 and warps % 8 == 0
    half, warps2 = busy(task_begin=nnz // 2)
    assert warps2 == warps and 0 < half < whole
