"""Failure detection without a GPU fault: a work-item cycle limit that runs
out makes the kernel abandon that job and return normally; the host reads
GP_ERR_TIMEOUT (or next_task = -1 for a time slice), other jobs of the same
launch finish exactly, and the context stays usable."""

import pytest

import oracle
from synth import named_pattern, workload_edges

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2009_10955_gb300 import native
    N = native()
    out = {}
    for name in ("rmat10", "er2000"):
        n, s, d = workload_edges(name)
        out[name] = (N.gp_graph_create_edges(s, d, n, N.GP_DEGREE_ORDER), oracle.build_csr(n, s, d))
    return N, out


def test_item_limit_abandons_and_context_survives(env):
    N, graphs = env
    g, _ = graphs["rmat10"]
    s = N.gp_schedule(N.gp_pattern_create(named_pattern("house")), g)
    with pytest.raises(N.GraphPiError) as e:
        N.gp_count(g, s, 0, N.make_opts(task_cycles=200))
    assert e.value.status == N.GP_ERR_TIMEOUT
    # same graph, same plan, no limit: exact count afterwards
    ge, re_ = graphs["er2000"]
    s2 = N.gp_schedule(N.gp_pattern_create(named_pattern("house")), ge)
    assert N.gp_count(ge, s2) == (N.GP_OK, oracle.count(named_pattern("house"), re_))


def test_time_slice_marks_only_the_abandoned_job(env):
    N, graphs = env
    gh, _ = graphs["rmat10"]
    gl, rl = graphs["er2000"]
    heavy = N.gp_schedule(N.gp_pattern_create(named_pattern("house")), gh)
    light = N.gp_schedule(N.gp_pattern_create(named_pattern("triangle")), gl)
    nl = gl.device_csr()[2]
    nh = gh.device_csr()[2]
    # the light (3-vertex) job runs one task per lane and has no inner loops,
    # so the limit only bites on the heavy job
    st, out, nxt = N.gp_count_batch_ranges([gh, gl], [heavy, light], [0, 0], [0, 0], [nh, nl],
                                           N.make_opts(task_cycles=200))
    assert nxt[0] == -1 and out[0] == 0
    assert nxt[1] == nl and int(out[1]) == oracle.count(named_pattern("triangle"), rl)
    assert st == N.GP_PARTIAL
