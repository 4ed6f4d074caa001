"""Inclusion-exclusion counting of the innermost loops (Section IV-D,
Algorithm 2), for kk = 2 to 5 replaced loops: every qualifying configuration
gives the oracle's count, stars also match their closed form
sum_v C(deg v, leaves), and partial counts (task ranges, budgets, time
slices) return undivided 128-bit totals that add up to the count times the
plan's divisor."""

import ctypes
from math import comb

import numpy as np
import pytest

import oracle
from oracle import planner_ref as pr
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
    for name, (n, m, seed) in {"er300": (300, 1500, 5), "er60": (60, 600, 9), "er30": (30, 300, 7)}.items():
        s, d = er_edges(n, m, seed)
        out[name] = (N.gp_graph_create_edges(s, d, n, N.GP_DEGREE_ORDER), oracle.build_csr(n, s, d))
    for name in ("rmat8", "er2000"):
        n, s, d = workload_edges(name)
        out[name] = (N.gp_graph_create_edges(s, d, n, N.GP_DEGREE_ORDER), oracle.build_csr(n, s, d))
    return N, out


@pytest.mark.parametrize("pname", ["house", "diamond", "tailed_triangle", "k6e", "c6chord", "grid3x2", "c5"])
def test_iep_every_configuration(env, pname):
    N, graphs = env
    g, ref = (graphs["er30"] if pname == "k6e" else
              graphs["er60"] if pname in ("c6chord", "grid3x2") else graphs["er300"])
    adj = named_pattern(pname)
    p = N.gp_pattern_create(adj)
    expect = oracle.count(adj, ref)
    scheds, _ = p.schedules()
    sets = p.restriction_sets()
    pairs = [(s, r) for s in scheds for r in sets]
    step = max(1, len(pairs) // 40)
    switched = 0
    for s, r in pairs[::step]:
        sc = N.gp_schedule_explicit(p, s, r)
        switched += sc.set_iep(True)
        assert N.gp_count(g, sc) == (N.GP_OK, expect), (s, r)
    if pname != "c5":   # every connected-prefix order of C5 ends in an adjacent pair: no IEP form
        assert switched > 0


@pytest.mark.parametrize("gname", ["rmat8", "er2000"])
def test_iep_top_plans(env, gname):
    N, graphs = env
    g, ref = graphs[gname]
    for pname in ("house", "diamond", "tailed_triangle"):
        adj = named_pattern(pname)
        sc = N.gp_schedule(N.gp_pattern_create(adj), g, top_k=3)
        plain = [N.gp_count(g, sc, i)[1] for i in range(len(sc))]
        sc.set_iep(True)
        iep = [N.gp_count(g, sc, i)[1] for i in range(len(sc))]
        assert plain == iep == [oracle.count(adj, ref)] * len(sc)


def test_iep_partial_count_needs_raw_total(env):
    N, graphs = env
    g, _ = graphs["er300"]
    sc = N.gp_schedule(N.gp_pattern_create(named_pattern("house")), g)
    assert sc.set_iep(True) == 1
    with pytest.raises(N.GraphPiError) as e:
        N.gp_count(g, sc, 0, N.make_opts(task_begin=0, task_end=10))
    assert e.value.status == N.GP_ERR_ARG
    st, raw = N.gp_count_raw(g, sc, 0, task_begin=0, task_end=10)
    assert st == N.GP_OK and raw >= 0


def star_count(ref, leaves):
    """Closed form: an L-leaf star is a centre and L of its neighbours."""
    deg = np.diff(ref.row_ptr)
    return sum(comb(int(d), leaves) for d in deg)


GENERAL = [("three_ears", 3), ("star5", 3), ("star6", 4), ("star7", 5)]


@pytest.mark.parametrize("pname,kk", GENERAL)
@pytest.mark.parametrize("gname", ["er300", "er2000", "rmat8"])
def test_iep_general_k_top_plans(env, pname, kk, gname):
    """The top plans with inclusion-exclusion over the innermost kk loops:
    the count equals the plain enumeration and the oracle (closed form for
    stars, whose enumeration on hub vertices is beyond the plain oracle)."""
    N, graphs = env
    g, ref = graphs[gname]
    adj = named_pattern(pname)
    sc = N.gp_schedule(N.gp_pattern_create(adj), g, top_k=3)
    plain = [N.gp_count(g, sc, i)[1] for i in range(len(sc))] if pname == "three_ears" else None
    assert sc.set_iep(True) >= 1
    assert max(sc.iep(i)[0] for i in range(len(sc))) == kk
    got = [N.gp_count(g, sc, i) for i in range(len(sc))]
    if pname.startswith("star"):
        expect = star_count(ref, int(pname[4:]) - 1)
        if gname == "er300":
            assert expect == oracle.count(adj, ref)
    else:
        expect = oracle.count(adj, ref)
        assert plain == [expect] * len(sc)
    assert got == [(N.GP_OK, expect)] * len(sc), (pname, gname, [sc.iep(i) for i in range(len(sc))])


@pytest.mark.parametrize("pname", ["three_ears", "star5", "star6", "path5"])
def test_iep_general_every_configuration(env, pname):
    """Sampled configurations (every efficient schedule x Algorithm 1 set)
    of patterns with three or more pairwise non-adjacent vertices last."""
    N, graphs = env
    g, ref = graphs["er60"]
    adj = named_pattern(pname)
    p = N.gp_pattern_create(adj)
    expect = oracle.count(adj, ref)
    scheds, _ = p.schedules()
    sets = p.restriction_sets()
    pairs = [(s, r) for s in scheds for r in sets]
    step = max(1, len(pairs) // 40)
    deep = 0
    for s, r in pairs[::step]:
        sc = N.gp_schedule_explicit(p, s, r)
        sc.set_iep(True)
        deep += sc.iep(0)[0] >= 3
        assert N.gp_count(g, sc) == (N.GP_OK, expect), (s, r, sc.iep(0))
    if pname != "path5":
        assert deep > 0


@pytest.mark.parametrize("pname", ["house", "three_ears", "star6"])
def test_iep_raw_totals_of_ranges_add_up(env, pname):
    """Task ranges and budgeted slices of an inclusion-exclusion plan: the
    undivided totals of disjoint ranges add up to count x divisor."""
    N, graphs = env
    g, ref = graphs["rmat8"]
    adj = named_pattern(pname)
    sc = N.gp_schedule(N.gp_pattern_create(adj), g)
    expect = N.gp_count(g, sc)[1]
    assert sc.set_iep(True) == 1
    kk, div = sc.iep(0)
    assert kk >= 2 and div >= 1
    assert N.gp_count(g, sc) == (N.GP_OK, expect)
    st, whole = N.gp_count_raw(g, sc)
    assert st == N.GP_OK and whole == expect * div
    nnz = g.device_csr()[2]
    cuts = [0, 1, 5, nnz // 3, nnz // 2 + 7, nnz - 1, nnz]
    parts = 0
    for a, b in zip(cuts[:-1], cuts[1:]):
        st, raw = N.gp_count_raw(g, sc, task_begin=a, task_end=b)
        assert st == N.GP_OK
        parts += raw
    assert parts == expect * div
    # budgeted slices, resumed where each stopped
    cur = ctypes.c_int64(0)
    acc, begin, rounds = 0, 0, 0
    while True:
        st, raw = N.gp_count_raw(g, sc, task_begin=begin, budget_cycles=100000, chunk=2,
                                 resume_cursor=ctypes.pointer(cur))
        acc += raw
        rounds += 1
        if st == N.GP_OK:
            break
        assert st == N.GP_PARTIAL and begin <= cur.value < nnz
        begin = cur.value
        assert rounds < 100000
    assert acc == expect * div
    # one time slice over several jobs: raw totals per job
    sp = N.gp_schedule(N.gp_pattern_create(named_pattern("diamond")), g)
    raw = np.zeros(4, dtype=np.uint64)
    st, out, nxt = N.gp_count_batch_ranges([g, g], [sc, sp], [0, 0], [0, 0], [0, 0], raw=raw)
    assert st == N.GP_OK and list(nxt) == [nnz, nnz]
    assert int(raw[0]) + (int(raw[1]) << 64) == expect * div and int(out[0]) == 0
    assert int(out[1]) == int(raw[2]) == N.gp_count(g, sp)[1] and int(raw[3]) == 0
