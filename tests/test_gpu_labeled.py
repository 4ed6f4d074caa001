"""Vertex-labelled patterns (NEXT: labelled extension): counts against the
oracle's labelled enumeration, listing agrees with the count, and uniform
labels reduce to the unlabelled count."""

import numpy as np
import pytest

import oracle
from synth import er_edges, named_pattern, workload_edges
from synth.rng import stream

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2009_10955_gb300 import native
    N = native()
    out = {}
    for name in ("er300", "rmat8"):
        if name == "er300":
            n = 300
            s, d = er_edges(n, 1500, 5)
        else:
            n, s, d = workload_edges(name)
        labels = (stream(99, 0, n) % np.uint64(3)).astype(np.int32)   # seeded labels 0..2
        g = N.gp_graph_create_edges(s, d, n, N.GP_DEGREE_ORDER)
        N.gp_graph_set_labels(g, labels)
        out[name] = (g, oracle.build_csr(n, s, d), labels)
    return N, out


CASES = [("triangle", [0, 1, 1]), ("c4", [0, 1, 0, 1]), ("house", [0, 0, 1, 1, 2]),
         ("path4", [2, 0, 0, 1]), ("diamond", [1, 1, 0, 0]), ("k4", [0, 0, 0, 1]), ("tailed_triangle", [0, 1, 1, 2])]


@pytest.mark.parametrize("gname", ["er300", "rmat8"])
@pytest.mark.parametrize("pname,plabels", CASES)
def test_labeled_count_and_list(env, gname, pname, plabels):
    import torch
    N, graphs = env
    g, ref, glabels = graphs[gname]
    adj = named_pattern(pname)
    sc = N.gp_schedule(N.gp_pattern_create_labeled(adj, plabels), g, top_k=2)
    expect = oracle.count_labeled(adj, plabels, ref, glabels)
    for i in range(len(sc)):
        assert N.gp_count(g, sc, i) == (N.GP_OK, expect)
    if expect < 2_000_000:
        k = adj.shape[0]
        buf = torch.empty((max(1, expect), k), dtype=torch.int32, device="cuda")
        st, n, nxt = N.gp_list(g, sc, 0, 0, 0, buf, max(1, expect))
        assert st == N.GP_OK and n == expect
        tup = buf[:n].cpu().numpy()
        perm = g.csr()[2]
        orig = perm[tup]                       # back to the input labelling
        assert np.all(glabels[orig] == np.array(plabels, dtype=np.int32)[None, :])


def test_uniform_labels_equal_unlabeled(env):
    N, graphs = env
    g, ref, _ = graphs["er300"]
    # a fresh graph with all labels equal
    n = 300
    s, d = er_edges(n, 1500, 5)
    gu = N.gp_graph_create_edges(s, d, n, N.GP_DEGREE_ORDER)
    N.gp_graph_set_labels(gu, np.zeros(n, np.int32))
    for pname in ("house", "c4", "k4"):
        adj = named_pattern(pname)
        lab = N.gp_count(gu, N.gp_schedule(N.gp_pattern_create_labeled(adj, [0] * adj.shape[0]), gu))
        plain = N.gp_count(gu, N.gp_schedule(N.gp_pattern_create(adj), gu))
        assert lab == plain == (N.GP_OK, oracle.count(adj, ref))


def test_labeled_plan_needs_graph_labels(env):
    N, _ = env
    n = 50
    s, d = er_edges(n, 200, 3)
    g = N.gp_graph_create_edges(s, d, n, N.GP_DEGREE_ORDER)
    sc = N.gp_schedule(N.gp_pattern_create_labeled(named_pattern("triangle"), [0, 0, 1]), g)
    with pytest.raises(N.GraphPiError) as e:
        N.gp_count(g, sc)
    assert e.value.status == N.GP_ERR_ARG
