"""GPU parity: the CUDA path (through the C ABI) against the oracle, on the
same seeded inputs. Counts are integers, so every comparison is exact."""

import numpy as np
import pytest

import oracle
from synth import named_pattern, er_edges, workload_edges, random_pattern_set

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def N():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2009_10955_gb300 import native
    return native()


_graphs = {}


def graph_pair(N, name, degree_order=True):
    """(device graph, oracle CSR in the same labelling) for a workload."""
    key = (name, degree_order)
    if key not in _graphs:
        if name.startswith("er:"):
            _, n, m, seed = name.split(":")
            n, m, seed = int(n), int(m), int(seed)
            s, d = er_edges(n, m, seed)
        else:
            n, s, d = workload_edges(name)
        g = N.gp_graph_create_edges(s, d, n, N.GP_DEGREE_ORDER if degree_order else 0)
        ref = oracle.build_csr(n, s, d)
        if degree_order:
            ref, _ = oracle.degree_relabel(ref)
        _graphs[key] = (g, ref)
    return _graphs[key]


# ------------------------------------------------------------------ graph build

@pytest.mark.parametrize("name", ["er2000", "rmat10", "rmat14", "cl10000", "er:1:0:1", "er:7:40:3"])
@pytest.mark.parametrize("degree_order", [False, True])
def test_csr_bit_exact(N, name, degree_order):
    g, ref = graph_pair(N, name, degree_order)
    row_ptr, col, perm = g.csr()
    assert np.array_equal(row_ptr, ref.row_ptr)
    assert np.array_equal(col, ref.col)
    st = g.stats(with_triangles=False)
    assert st["n"] == ref.n and st["m"] == ref.nnz // 2
    assert st["max_deg"] == (int(np.diff(ref.row_ptr).max()) if ref.n else 0)


def test_csr_from_csr_input(N):
    n, s, d = workload_edges("rmat10")
    ref = oracle.build_csr(n, s, d)
    g = N.gp_graph_create_csr(ref.row_ptr, ref.col, n, 0)
    rp, col, _ = g.csr()
    assert np.array_equal(rp, ref.row_ptr) and np.array_equal(col, ref.col)
    g2 = N.gp_graph_create_csr(ref.row_ptr, ref.col, n, N.GP_ASSUME_CLEAN)
    rp2, col2, _ = g2.csr()
    assert np.array_equal(rp2, ref.row_ptr) and np.array_equal(col2, ref.col)


def test_graph_bad_ids_rejected(N):
    with pytest.raises(N.GraphPiError) as e:
        N.gp_graph_create_edges(np.array([0, 5], np.int32), np.array([1, 2], np.int32), 5)
    assert e.value.status == N.GP_ERR_ARG


def test_triangle_stat_matches_oracle(N):
    for name in ["er2000", "rmat12", "cl10000"]:
        g, ref = graph_pair(N, name)
        assert g.stats()["tri_cnt"] == 6 * oracle.triangles(ref)


# ------------------------------------------------------------------ counts

SMALL = ["er2000", "rmat8", "er:300:1500:5", "er:57:400:9"]
P5 = ["triangle", "path3", "k4", "c4", "diamond", "tailed_triangle", "star4", "house", "c5", "k5", "path5"]


@pytest.mark.parametrize("gname", SMALL)
@pytest.mark.parametrize("pname", P5)
def test_count_matches_oracle(N, gname, pname):
    g, ref = graph_pair(N, gname)
    adj = named_pattern(pname)
    p = N.gp_pattern_create(adj)
    s = N.gp_schedule(p, g, top_k=3)
    expect = oracle.count(adj, ref)
    for i in range(len(s)):
        st, c = N.gp_count(g, s, i)
        assert st == N.GP_OK and c == expect, (pname, gname, i, s.get(i))


@pytest.mark.parametrize("pname", ["k6e", "c6chord", "grid3x2", "c6", "k6"])
def test_six_vertex_patterns(N, pname):
    g, ref = graph_pair(N, "er:57:400:9")
    adj = named_pattern(pname)
    expect = oracle.count(adj, ref)
    s = N.gp_schedule(N.gp_pattern_create(adj), g, top_k=3)
    for i in range(len(s)):
        assert N.gp_count(g, s, i) == (N.GP_OK, expect)


@pytest.mark.parametrize("pname", ["c7", "k7"])
def test_seven_vertex_patterns(N, pname):
    g, ref = graph_pair(N, "er:20:120:4")
    adj = named_pattern(pname)
    s = N.gp_schedule(N.gp_pattern_create(adj), g, top_k=2)
    expect = oracle.count(adj, ref)
    for i in range(len(s)):
        assert N.gp_count(g, s, i) == (N.GP_OK, expect)


@pytest.mark.parametrize("pname", ["house", "c4", "diamond", "tailed_triangle", "k4", "c5"])
def test_every_configuration_agrees(N, pname):
    """All efficient schedules x all restriction sets give the oracle count
    (the restricted count times |Aut| is the unrestricted count)."""
    g, ref = graph_pair(N, "er:300:1500:5")
    adj = named_pattern(pname)
    p = N.gp_pattern_create(adj)
    expect = oracle.count(adj, ref)
    scheds, _ = p.schedules()
    sets = p.restriction_sets()
    pairs = [(s, r) for s in scheds for r in sets]
    step = max(1, len(pairs) // 60)
    for s, r in pairs[::step]:
        sc = N.gp_schedule_explicit(p, s, r)
        assert N.gp_count(g, sc) == (N.GP_OK, expect), (s, r)


@pytest.mark.parametrize("gname", ["er:300:1500:5", "rmat10"])
@pytest.mark.parametrize("pname", ["c4", "c5", "house", "diamond", "tailed_triangle", "k4", "path4", "k5",
                                   "k6e", "k6", "k7"])
def test_bitmap_paths_equal_list_path(N, gname, pname):
    """Every sampled configuration: the core bit-matrix paths (default, with
    the three-level lane tail where the plan allows it; one candidate per
    warp; one candidate per lane for the last two levels) give the count of
    the pure list path, which equals the oracle's."""
    g, ref = graph_pair(N, gname)
    adj = named_pattern(pname)
    p = N.gp_pattern_create(adj)
    scheds, _ = p.schedules()
    sets = p.restriction_sets()
    pairs = [(sc, r) for sc in scheds for r in sets]
    step = max(1, len(pairs) // 150)
    expect = None
    for sc, r in pairs[::step]:
        one = N.gp_schedule_explicit(p, sc, r)
        lists = N.gp_count(g, one, 0, N.make_opts(flags=N.GP_COUNT_NO_CORE))
        assert N.gp_count(g, one) == lists, (sc, r)
        assert N.gp_count(g, one, 0, N.make_opts(flags=N.GP_COUNT_WARP_BITMAP)) == lists, (sc, r)
        assert N.gp_count(g, one, 0, N.make_opts(flags=N.GP_COUNT_LANE_BITMAP)) == lists, (sc, r)
        if expect is None:
            expect = lists
        assert lists == expect, (sc, r)
    if gname.startswith("er") or pname in ("c4", "k4", "diamond", "tailed_triangle", "path4"):
        assert expect[1] == oracle.count(adj, ref)


def test_random_patterns_batched_equals_single_and_oracle(N):
    g, ref = graph_pair(N, "er:300:1500:5")
    pats = random_pattern_set(16, 3, 6, 0.5, seed=11)
    scheds = [N.gp_schedule(N.gp_pattern_create(a), g, top_k=2) for a in pats]
    graphs, ss, idx = [], [], []
    for s in scheds:
        for i in range(len(s)):
            graphs.append(g); ss.append(s); idx.append(i)
    batched = N.gp_count_batch(graphs, ss, idx)
    for j, (s, i) in enumerate(zip(ss, idx)):
        st, single = N.gp_count(g, s, i)
        assert single == int(batched[j])
    for a, s in zip(pats, scheds):
        expect = oracle.count(a, ref)
        assert N.gp_count(g, s, 0)[1] == expect


def test_batch_across_graphs(N):
    ga, ra = graph_pair(N, "er2000")
    gb, rb = graph_pair(N, "rmat8")
    adj = named_pattern("house")
    p = N.gp_pattern_create(adj)
    sa, sb = N.gp_schedule(p, ga), N.gp_schedule(p, gb)
    out = N.gp_count_batch([ga, gb, ga], [sa, sb, sa], [0, 0, 0])
    assert list(out) == [oracle.count(adj, ra), oracle.count(adj, rb), oracle.count(adj, ra)]


@pytest.mark.parametrize("pname", ["k4", "triangle", "k5"])
def test_partial_core_graph(N, pname):
    """A graph larger than the 8192-vertex core: tasks whose second vertex
    is a core vertex run on the bit matrix, the others on lists. Whole
    counts against the restricted oracle (k4, triangle); for k5, whole
    counts with and without the bit matrix, and sampled roots against the
    oracle."""
    g, ref = graph_pair(N, "rmat14")
    adj = named_pattern(pname)
    s = N.gp_schedule(N.gp_pattern_create(adj), g)
    order, res, _ = s.get(0)
    got = N.gp_count(g, s)
    no_core = N.gp_count(g, s, 0, N.make_opts(flags=N.GP_COUNT_NO_CORE))
    assert got == no_core
    for split in (2, 8, 33):           # high-degree tasks cut into parts
        assert N.gp_count(g, s, 0, N.make_opts(split=split)) == got
        assert N.gp_count(g, s, 0, N.make_opts(split=split, flags=N.GP_COUNT_NO_CORE)) == got
        for f in (N.GP_COUNT_LANE_BITMAP, N.GP_COUNT_WARP_BITMAP):
            assert N.gp_count(g, s, 0, N.make_opts(split=split, flags=f)) == got
    if pname != "k5":
        assert got[1] == oracle.count_restricted(adj, order, res, ref)
    else:
        for r in [1, 7, 40, 300, 2000, 8191, 8192, 9000, 12000]:
            o = N.make_opts(task_begin=int(ref.row_ptr[r]), task_end=int(ref.row_ptr[r + 1]))
            expect = oracle.count_restricted(adj, order, res, ref, root_begin=r, root_end=r + 1)
            assert N.gp_count(g, s, 0, o)[1] == expect, r


@pytest.mark.parametrize("pname", ["house", "diamond", "c4"])
def test_split_tasks_agree(N, pname):
    g, ref = graph_pair(N, "rmat12")
    s = N.gp_schedule(N.gp_pattern_create(named_pattern(pname)), g, top_k=2)
    for i in range(len(s)):
        base = N.gp_count(g, s, i)
        for split in (3, 16):
            assert N.gp_count(g, s, i, N.make_opts(split=split)) == base


def test_degree_order_invariance(N):
    for name in ["rmat10", "er2000"]:
        g1, _ = graph_pair(N, name, degree_order=True)
        g0, _ = graph_pair(N, name, degree_order=False)
        for pname in ["house", "k4", "c4"]:
            p = N.gp_pattern_create(named_pattern(pname))
            assert N.gp_count(g1, N.gp_schedule(p, g1))[1] == N.gp_count(g0, N.gp_schedule(p, g0))[1]


# ------------------------------------------------------------------ edge cases

def test_empty_and_degenerate_graphs(N):
    tri = N.gp_pattern_create(named_pattern("triangle"))
    house = N.gp_pattern_create(named_pattern("house"))
    cases = [
        (0, [], []),                           # no vertices
        (5, [], []),                           # isolated vertices
        (4, [1, 2, 3], [1, 2, 3]),             # self loops only
        (2, [0], [1]),                         # one edge
        (8, [0] * 7, list(range(1, 8))),       # star: no triangle
    ]
    for n, s, d in cases:
        g = N.gp_graph_create_edges(np.array(s, np.int32), np.array(d, np.int32), n, N.GP_DEGREE_ORDER)
        for p in (tri, house):
            assert N.gp_count(g, N.gp_schedule(p, g)) == (N.GP_OK, 0)


def test_task_ranges_and_resume_sum_to_total(N):
    g, ref = graph_pair(N, "rmat10")
    p = N.gp_pattern_create(named_pattern("house"))
    s = N.gp_schedule(p, g)
    total = N.gp_count(g, s)[1]
    nnz = g.device_csr()[2]
    cuts = [0, 1, 7, nnz // 3, nnz // 2 + 5, nnz - 1, nnz]
    parts = 0
    for a, b in zip(cuts[:-1], cuts[1:]):
        st, c = N.gp_count(g, s, 0, N.make_opts(task_begin=a, task_end=b))
        assert st == N.GP_OK
        parts += c
    assert parts == total


def test_budget_partial_then_resume(N):
    import ctypes
    g, _ = graph_pair(N, "rmat12")
    p = N.gp_pattern_create(named_pattern("house"))
    s = N.gp_schedule(p, g)
    total = N.gp_count(g, s)[1]
    cur = ctypes.c_int64(0)
    acc, begin, rounds = 0, 0, 0
    nnz = g.device_csr()[2]
    while True:
        o = N.make_opts(task_begin=begin, budget_cycles=200000, chunk=4,
                        resume_cursor=ctypes.pointer(cur))
        st, c = N.gp_count(g, s, 0, o)
        acc += c
        rounds += 1
        if st == N.GP_OK:
            break
        assert st == N.GP_PARTIAL and begin <= cur.value < nnz
        begin = cur.value
        assert rounds < 100000
    assert acc == total


# ------------------------------------------------------------ full-size samples

def _sampled_rows(ref, count, seed):
    deg = np.diff(ref.row_ptr)
    rng = np.random.default_rng(seed)
    nz = np.nonzero(deg)[0]
    pick = set(rng.choice(nz, size=min(count, len(nz)), replace=False).tolist())
    pick.add(int(nz[-1]))            # the lowest-degree non-isolated vertex
    return sorted(pick)


@pytest.mark.parametrize("pname", ["triangle", "k4", "house", "k5", "diamond"])
def test_rmat20_sampled_roots(N, pname):
    """Full-size R-MAT scale-20 graph: the CSR is bit-exact, and for sampled
    root vertices the count of the tasks rooted there equals the oracle's
    restricted enumeration from the same roots with the same plan."""
    g, ref = graph_pair(N, "rmat20")
    rp, col, _ = g.csr()
    assert np.array_equal(rp, ref.row_ptr) and np.array_equal(col, ref.col)
    adj = named_pattern(pname)
    s = N.gp_schedule(N.gp_pattern_create(adj), g)
    order, res, _ = s.get(0)
    deg = np.diff(ref.row_ptr)
    rows = [r for r in _sampled_rows(ref, 24, seed=1) if deg[r] <= 2000][:16]
    for r in rows:
        o = N.make_opts(task_begin=int(ref.row_ptr[r]), task_end=int(ref.row_ptr[r + 1]))
        st, c = N.gp_count(g, s, 0, o)
        expect = oracle.count_restricted(adj, order, res, ref, root_begin=r, root_end=r + 1)
        assert c == expect, (pname, r, int(deg[r]))


@pytest.mark.parametrize("pname,roots", [("k6e", None), ("c6chord", [(9700, 10000), (2000, 2050)]),
                                         ("grid3x2", [(9700, 10000), (2000, 2050)])])
def test_chung_lu_six_vertex_patterns(N, pname, roots):
    """The Chung-Lu workload's 6-vertex patterns on the same generator at
    10,000 vertices (exponent 2.1, mean degree 17.5): the whole K6-e count,
    and the counts of two root ranges (lowest-degree roots, and roots of
    degree about 16) for the 6-cycle with a chord and the 3x2 grid, against
    the oracle's restricted enumeration with the same plan."""
    g, ref = graph_pair(N, "cl10000")
    adj = named_pattern(pname)
    # the plan ranked first under the library's default graph statistics
    # (fixed, so that the oracle's share of the test stays within a minute)
    s = N.gp_schedule(N.gp_pattern_create(adj), None)
    order, res, _ = s.get(0)
    if roots is None:
        assert N.gp_count(g, s) == (N.GP_OK, oracle.count_restricted(adj, order, res, ref))
        return
    for lo, hi in roots:
        o = N.make_opts(task_begin=int(ref.row_ptr[lo]), task_end=int(ref.row_ptr[hi]))
        expect = oracle.count_restricted(adj, order, res, ref, root_begin=lo, root_end=hi)
        assert N.gp_count(g, s, 0, o) == (N.GP_OK, expect), (pname, lo, hi)


def test_chung_lu_4m_sampled_roots(N):
    """Full-size Chung-Lu workload (4,000,000 vertices): the CSR is
    bit-exact, and for sampled roots the K6-e count of the tasks rooted
    there equals the oracle's restricted enumeration with the same plan."""
    g, ref = graph_pair(N, "cl4m")
    rp, col, _ = g.csr()
    assert np.array_equal(rp, ref.row_ptr) and np.array_equal(col, ref.col)
    adj = named_pattern("k6e")
    s = N.gp_schedule(N.gp_pattern_create(adj), g)
    order, res, _ = s.get(0)
    deg = np.diff(ref.row_ptr)
    rows = [r for r in _sampled_rows(ref, 24, seed=1) if deg[r] <= 2000][:16]
    for r in rows:
        o = N.make_opts(task_begin=int(ref.row_ptr[r]), task_end=int(ref.row_ptr[r + 1]))
        st, c = N.gp_count(g, s, 0, o)
        expect = oracle.count_restricted(adj, order, res, ref, root_begin=r, root_end=r + 1)
        assert c == expect, (r, int(deg[r]))


# ----------------------------------------------- full-size hub roots, whole counts

ORACLE_LEAVES_PER_WINDOW = 300_000_000     # keeps each oracle call within seconds


def _hub_windows(N, g, s, ref, roots, width=64):
    """CSR entry windows inside the rows of high-degree roots (their first,
    middle and last `width` entries), each narrowed from its start until the
    GPU count of the window is small enough for the oracle's enumeration,
    which visits every embedding one by one."""
    out = []
    for r in roots:
        b, e = int(ref.row_ptr[r]), int(ref.row_ptr[r + 1])
        for a in sorted({b, max(b, (b + e) // 2 - width // 2), max(b, e - width)}):
            z = min(e, a + width)
            while z > a:
                c = N.gp_count(g, s, 0, N.make_opts(task_begin=a, task_end=z))[1]
                if c <= ORACLE_LEAVES_PER_WINDOW:
                    out.append((r, a, z, c))
                    break
                z = a + (z - a) // 2
    return out


def _hub_roots(ref, extra, seed):
    deg = np.diff(ref.row_ptr)
    big = np.nonzero(deg > 2000)[0]
    rng = np.random.default_rng(seed)
    pick = [0, 1, 2] + sorted(rng.choice(big[3:], size=min(extra, max(0, len(big) - 3)), replace=False).tolist())
    return pick, deg


@pytest.mark.parametrize("pname", ["triangle", "k4", "house", "k5", "diamond"])
def test_rmat20_hub_roots(N, pname):
    """Full-size R-MAT scale 20, roots of degree > 2000 (the three highest
    and two sampled): windows of their edge tasks, counted whole and with
    every task cut into 8 parts (the split heavy prefix), equal the oracle's
    restricted enumeration of the same CSR entries with the same plan."""
    g, ref = graph_pair(N, "rmat20")
    adj = named_pattern(pname)
    s = N.gp_schedule(N.gp_pattern_create(adj), g)
    order, res, _ = s.get(0)
    roots, deg = _hub_roots(ref, 2, seed=7)
    wins = _hub_windows(N, g, s, ref, roots)
    assert len({r for r, *_ in wins}) >= 4, wins
    for r, a, z, c in wins:
        assert deg[r] > 2000
        expect = oracle.count_restricted_entries(adj, order, res, ref, a, z)
        assert c == expect, (pname, r, a, z)
        for split in (8,):
            assert N.gp_count(g, s, 0, N.make_opts(task_begin=a, task_end=z, split=split)) == (N.GP_OK, expect)


def test_chung_lu_4m_hub_roots(N):
    """Full-size Chung-Lu workload: K6-e over windows of the edge tasks of
    roots of degree > 2000, whole and split, against the oracle."""
    g, ref = graph_pair(N, "cl4m")
    adj = named_pattern("k6e")
    s = N.gp_schedule(N.gp_pattern_create(adj), g)
    order, res, _ = s.get(0)
    roots, deg = _hub_roots(ref, 2, seed=8)
    wins = _hub_windows(N, g, s, ref, roots)
    assert len({r for r, *_ in wins}) >= 4, wins
    for r, a, z, c in wins:
        assert deg[r] > 2000
        expect = oracle.count_restricted_entries(adj, order, res, ref, a, z)
        assert c == expect, (r, a, z)
        assert N.gp_count(g, s, 0, N.make_opts(task_begin=a, task_end=z, split=8)) == (N.GP_OK, expect)


@pytest.mark.parametrize("pname", ["triangle", "k4", "k5"])
def test_rmat20_whole_counts_agree_across_plans_and_paths(N, pname):
    """Full-size whole counts the oracle cannot finish: the three plans the
    model ranks first, the list path alone (no core bit matrix), the three
    bitmap-subtree variants and split heavy tasks all give one count."""
    g, _ = graph_pair(N, "rmat20")
    s = N.gp_schedule(N.gp_pattern_create(named_pattern(pname)), g, top_k=3)
    base = N.gp_count(g, s, 0)
    assert base[0] == N.GP_OK and base[1] > 0
    for i in range(1, len(s)):
        assert N.gp_count(g, s, i) == base, i
    for f in (N.GP_COUNT_NO_CORE, N.GP_COUNT_WARP_BITMAP, N.GP_COUNT_LANE_BITMAP):
        assert N.gp_count(g, s, 0, N.make_opts(flags=f)) == base, f
    assert N.gp_count(g, s, 0, N.make_opts(split=8)) == base


def test_chung_lu_4m_whole_k6e_agrees_across_plans_and_paths(N):
    """Full-size K6-e on the Chung-Lu workload: the top three plans, the
    list path without the core bit matrix, inclusion-exclusion over the
    last two loops and split heavy tasks give one count."""
    g, _ = graph_pair(N, "cl4m")
    adj = named_pattern("k6e")
    s = N.gp_schedule(N.gp_pattern_create(adj), g, top_k=3)
    base = N.gp_count(g, s, 0)
    assert base[0] == N.GP_OK and base[1] > 0
    for i in range(1, len(s)):
        assert N.gp_count(g, s, i) == base, i
    assert N.gp_count(g, s, 0, N.make_opts(flags=N.GP_COUNT_NO_CORE)) == base
    assert N.gp_count(g, s, 0, N.make_opts(split=8)) == base
    si = N.gp_schedule(N.gp_pattern_create(adj), g)
    assert si.set_iep(True) == 1
    assert N.gp_count(g, si, 0) == base


@pytest.mark.parametrize("pname", ["k6", "k7"])
def test_large_cliques_on_a_full_core(N, pname):
    """Six- and seven-vertex cliques on a graph whose core bit matrix is full
    (8,192 vertices, 256 words a row): the bitmap subtree then needs 40 and
    48 KB of shared memory per block, beside the kernel's own; every bitmap
    variant must launch and equal the list path."""
    g, _ = graph_pair(N, "rmat14")
    s = N.gp_schedule(N.gp_pattern_create(named_pattern(pname)), g)
    lists = N.gp_count(g, s, 0, N.make_opts(flags=N.GP_COUNT_NO_CORE))
    assert lists[0] == N.GP_OK
    for f in (0, N.GP_COUNT_WARP_BITMAP, N.GP_COUNT_LANE_BITMAP):
        assert N.gp_count(g, s, 0, N.make_opts(flags=f)) == lists, f
