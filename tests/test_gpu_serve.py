"""Continuous-batching server: requests that arrive while others run are
admitted between time slices, and every request's count is the same alone
and in the mix (and equals the oracle)."""

import time

import numpy as np
import pytest

import oracle
from synth import named_pattern, random_pattern_set, workload_edges

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2009_10955_gb300 import native
    N = native()
    graphs, refs = {}, {}
    for name in ("rmat8", "rmat10", "er2000"):
        n, s, d = workload_edges(name)
        graphs[name] = N.gp_graph_create_edges(s, d, n, N.GP_DEGREE_ORDER)
        refs[name] = oracle.build_csr(n, s, d)
    return N, graphs, refs


def test_alone_equals_mixed_equals_oracle(env):
    from paper_2009_10955_gb300.serve import Server
    N, graphs, refs = env
    pats = random_pattern_set(12, 3, 5, 0.5, seed=3) + [named_pattern("house"), named_pattern("k4")]
    names = list(graphs)
    reqs = [(names[i % len(names)], p) for i, p in enumerate(pats)]
    # alone: one request at a time through the server
    srv = Server(graphs, slice_ms=2.0)
    alone = []
    for gname, adj in reqs:
        r = srv.submit(gname, adj)
        assert r.done.wait(120)
        assert r.error is None, r.error
        alone.append(r.count)
    srv.close()
    # mixed: all at once, with short slices so that jobs span several slices
    srv = Server(graphs, slice_ms=0.2)
    rs = [srv.submit(g, a) for g, a in reqs]
    for r in rs:
        assert r.done.wait(300)
        assert r.error is None, r.error
    srv.close()
    mixed = [r.count for r in rs]
    assert mixed == alone
    for (gname, adj), c in zip(reqs, mixed):
        assert c == oracle.count(adj, refs[gname])
    assert srv.slices >= 1


def test_late_arrivals_join_running_batch(env):
    from paper_2009_10955_gb300.serve import Server
    N, graphs, refs = env
    srv = Server(graphs, slice_ms=0.5)
    first = srv.submit("rmat8", named_pattern("house"))
    time.sleep(0.01)
    late = [srv.submit("er2000", named_pattern("c4")), srv.submit("rmat8", named_pattern("k4"))]
    for r in [first] + late:
        assert r.done.wait(120) and r.error is None
    srv.close()
    assert first.count == oracle.count(named_pattern("house"), refs["rmat8"])
    assert late[0].count == oracle.count(named_pattern("c4"), refs["er2000"])
    assert late[1].count == oracle.count(named_pattern("k4"), refs["rmat8"])


def test_bad_request_is_answered_with_error(env):
    from paper_2009_10955_gb300.serve import Server
    N, graphs, _ = env
    srv = Server(graphs)
    bad = np.zeros((3, 3), np.uint8)                     # not connected
    r = srv.submit("rmat8", bad)
    assert r.done.wait(30)
    assert r.error is not None and r.count is None
    ok = srv.submit("rmat8", named_pattern("triangle"))
    assert ok.done.wait(30) and ok.error is None
    srv.close()
