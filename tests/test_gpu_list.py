"""Listing mode (NEXT: emit the embeddings): the tuples the GPU writes are
exactly the oracle's restricted enumeration for the same plan, as many as
the count, and capacity-limited calls resume without loss or repetition."""

import numpy as np
import pytest

import oracle
from synth import er_edges, named_pattern, workload_edges

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2009_10955_gb300 import native
    N = native()
    out = {}
    s, d = er_edges(300, 1500, 5)
    out["er300"] = (N.gp_graph_create_edges(s, d, 300, N.GP_DEGREE_ORDER),
                    oracle.degree_relabel(oracle.build_csr(300, s, d))[0])
    n, s, d = workload_edges("rmat8")
    out["rmat8"] = (N.gp_graph_create_edges(s, d, n, N.GP_DEGREE_ORDER),
                    oracle.degree_relabel(oracle.build_csr(n, s, d))[0])
    return N, out


def list_all(N, g, sc, k, capacity):
    import torch
    nnz = g.device_csr()[2]
    buf = torch.empty((max(1, capacity), k), dtype=torch.int32, device="cuda")
    chunks, begin = [], 0
    while True:
        st, n, nxt = N.gp_list(g, sc, 0, begin, nnz, buf, capacity)
        chunks.append(buf[:n].cpu().numpy().copy())
        assert nxt > begin or nxt == nnz
        begin = nxt
        if st == N.GP_OK:
            break
        assert st == N.GP_PARTIAL
    return np.concatenate(chunks) if chunks else np.zeros((0, k), np.int32)


@pytest.mark.parametrize("gname", ["er300", "rmat8"])
@pytest.mark.parametrize("pname", ["triangle", "c4", "house", "k4", "diamond", "tailed_triangle", "path4", "c5"])
def test_listing_equals_oracle_and_count(env, gname, pname):
    N, graphs = env
    g, ref = graphs[gname]
    adj = named_pattern(pname)
    k = adj.shape[0]
    sc = N.gp_schedule(N.gp_pattern_create(adj), g)
    order, res, _ = sc.get(0)
    count = N.gp_count(g, sc)[1]
    if count > 4_000_000:
        pytest.skip("too many embeddings to compare tuple by tuple")
    full = list_all(N, g, sc, k, count + 1)
    assert len(full) == count
    expect, total = oracle.list_restricted(adj, order, res, ref, cap=count + 1)
    assert total == count

    def canon(a):
        return a[np.lexsort(a.T[::-1])] if len(a) else a
    assert np.array_equal(canon(full), canon(expect))
    # every tuple is an embedding: pattern edges map to graph edges
    rows = [set(ref.col[ref.row_ptr[u]:ref.row_ptr[u + 1]].tolist()) for u in range(ref.n)]
    for t in full[:2000]:
        for a in range(k):
            for b in range(k):
                if adj[a, b]:
                    assert int(t[b]) in rows[int(t[a])]
    # back-pressure: small buffers, same tuples in the same order
    if count > 10:
        import torch
        try:
            chunked = list_all(N, g, sc, k, count // 4 + 1)
        except N.GraphPiError as e:
            assert e.status == N.GP_ERR_SCRATCH      # one task alone exceeds the buffer
        else:
            assert np.array_equal(chunked, full)


def test_listing_rejects_iep_plans(env):
    import torch
    N, graphs = env
    g, _ = graphs["er300"]
    sc = N.gp_schedule(N.gp_pattern_create(named_pattern("house")), g)
    assert sc.set_iep(True) == 1
    buf = torch.empty((10, 5), dtype=torch.int32, device="cuda")
    with pytest.raises(N.GraphPiError) as e:
        N.gp_list(g, sc, 0, 0, 0, buf, 10)
    assert e.value.status == N.GP_ERR_ARG
