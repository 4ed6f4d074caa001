"""Pins for the oracle: closed forms, brute force over vertex tuples, and the
values the paper prints. None of these re-derive a result from the oracle
itself; each is fixed by mathematics or by the paper's text."""

import itertools
import math

import numpy as np
import pytest

import oracle
from oracle import planner_ref as pr
from synth import named_pattern, edges_to_adj, er_edges


# ---------------------------------------------------------------- helpers

def complete(n):
    s, d = zip(*[(a, b) for a in range(n) for b in range(a + 1, n)])
    return oracle.build_csr(n, np.array(s), np.array(d))


def from_edges(n, edges):
    s, d = zip(*edges)
    return oracle.build_csr(n, np.array(s), np.array(d))


def cycle_graph(n):
    return from_edges(n, [(i, (i + 1) % n) for i in range(n)])


def bipartite(a, b):
    return from_edges(a + b, [(i, a + j) for i in range(a) for j in range(b)])


def petersen():
    outer = [(i, (i + 1) % 5) for i in range(5)]
    spokes = [(i, i + 5) for i in range(5)]
    inner = [(5 + i, 5 + (i + 2) % 5) for i in range(5)]
    return from_edges(10, outer + spokes + inner)


def brute_force_maps(pattern, gadj):
    """All injective k-tuples of graph vertices that keep every pattern edge."""
    k = pattern.shape[0]
    n = gadj.shape[0]
    pe = [(a, b) for a in range(k) for b in range(k) if pattern[a, b]]
    return sum(1 for t in itertools.permutations(range(n), k)
               if all(gadj[t[a], t[b]] for a, b in pe))


def brute_force_aut(pattern):
    k = pattern.shape[0]
    return sum(1 for p in itertools.permutations(range(k))
               if all(pattern[p[a], p[b]] for a in range(k) for b in range(k) if pattern[a, b]))


def dense(g):
    a = np.zeros((g.n, g.n), dtype=np.uint8)
    for u in range(g.n):
        a[u, g.col[g.row_ptr[u]:g.row_ptr[u + 1]]] = 1
    return a


# ------------------------------------------------------------------- CSR

def test_csr_matches_set_definition():
    n = 50
    s, d = er_edges(n, 400, seed=7)
    s = np.concatenate([s, [3, 3, 9]]).astype(np.int32)      # a self loop and a duplicate
    d = np.concatenate([d, [3, 9, 3]]).astype(np.int32)
    g = oracle.build_csr(n, s, d)
    expect = {u: sorted({int(b) for a, b in zip(s, d) if a == u and a != b} |
                        {int(a) for a, b in zip(s, d) if b == u and a != b}) for u in range(n)}
    for u in range(n):
        assert list(g.col[g.row_ptr[u]:g.row_ptr[u + 1]]) == expect[u]
    assert g.nnz == sum(len(v) for v in expect.values())


def test_csr_empty_and_isolated():
    g = oracle.build_csr(5, np.zeros(0, np.int32), np.zeros(0, np.int32))
    assert g.nnz == 0 and list(g.row_ptr) == [0] * 6
    g = oracle.build_csr(4, np.array([2, 2]), np.array([2, 2]))   # only self loops
    assert g.nnz == 0


# -------------------------------------------------------- automorphisms

def test_aut_k7_is_5040():
    # Section II-B: each 7-clique embedding has 5,040 automorphisms.
    assert oracle.aut_count(named_pattern("k7")) == 5040
    assert len(pr.automorphisms(named_pattern("k7").tolist())) == 5040


@pytest.mark.parametrize("k", [3, 4, 5, 6])
def test_aut_closed_forms(k):
    assert oracle.aut_count(named_pattern({3: "triangle", 4: "k4", 5: "k5", 6: "k6"}[k])) == math.factorial(k)
    cyc = edges_to_adj(k, [(i, (i + 1) % k) for i in range(k)])
    assert oracle.aut_count(cyc) == 2 * k                       # dihedral group
    star = edges_to_adj(k, [(0, i) for i in range(1, k)])
    assert oracle.aut_count(star) == math.factorial(k - 1)
    path = edges_to_adj(k, [(i, i + 1) for i in range(k - 1)])
    assert oracle.aut_count(path) == 2


def test_aut_rectangle_contains_b_d_swap():
    # Section IV-A: the rectangle's group contains (A)(B,D)(C).
    c4 = named_pattern("c4").tolist()
    auts = pr.automorphisms(c4)
    assert len(auts) == 8
    assert (0, 3, 2, 1) in auts
    assert oracle.aut_count(named_pattern("c4")) == 8


@pytest.mark.parametrize("name", ["house", "c6chord", "grid3x2", "k6e", "tailed_triangle", "diamond"])
def test_aut_brute_force(name):
    p = named_pattern(name)
    assert oracle.aut_count(p) == brute_force_aut(p) == len(pr.automorphisms(p.tolist()))


# -------------------------------------------------------------- closed forms

@pytest.mark.parametrize("n", [5, 7, 9])
def test_cliques_in_complete_graph(n):
    g = complete(n)
    for k, name in [(3, "triangle"), (4, "k4"), (5, "k5")]:
        assert oracle.count(named_pattern(name), g) == math.comb(n, k)


@pytest.mark.parametrize("n", [5, 7, 8])
def test_house_and_cycles_in_complete_graph(n):
    g = complete(n)
    assert oracle.count(named_pattern("house"), g) == n * (n - 1) * (n - 2) * (n - 3) * (n - 4) // 2
    for k in (4, 5, 6):
        if k <= n:
            expect = math.factorial(n) // (math.factorial(n - k) * 2 * k)
            assert oracle.count(named_pattern(f"c{k}"), g) == expect


@pytest.mark.parametrize("n", [6, 7, 9])
def test_ring_has_one_n_cycle_and_no_shorter(n):
    g = cycle_graph(n)
    if n <= 7:
        assert oracle.count(named_pattern(f"c{n}"), g) == 1
    for k in range(3, min(n, 8)):
        if k < n:
            cyc = edges_to_adj(k, [(i, (i + 1) % k) for i in range(k)])
            assert oracle.count(cyc, g) == 0
    # paths with k vertices on an n-ring: n of them (one per starting edge)
    for k in (3, 4, 5):
        assert oracle.count(named_pattern(f"path{k}"), g) == n


@pytest.mark.parametrize("a,b", [(2, 3), (3, 3), (3, 4), (4, 5)])
def test_even_cycles_in_complete_bipartite(a, b):
    g = bipartite(a, b)
    for l in (2, 3):
        if 2 * l <= 7:
            expect = math.comb(a, l) * math.comb(b, l) * math.factorial(l) ** 2 // (2 * l)
            cyc = edges_to_adj(2 * l, [(i, (i + 1) % (2 * l)) for i in range(2 * l)])
            assert oracle.count(cyc, g) == expect
    assert oracle.count(named_pattern("triangle"), g) == 0


def test_star_has_no_triangles_and_known_stars():
    g = from_edges(8, [(0, i) for i in range(1, 8)])
    assert oracle.count(named_pattern("triangle"), g) == 0
    assert oracle.triangles(g) == 0
    assert oracle.count(named_pattern("star4"), g) == math.comb(7, 3)


def test_petersen_cycles():
    # The Petersen graph has girth 5, 12 pentagons and 10 hexagons.
    g = petersen()
    assert oracle.count(named_pattern("triangle"), g) == 0
    assert oracle.count(named_pattern("c4"), g) == 0
    assert oracle.count(named_pattern("c5"), g) == 12
    assert oracle.count(named_pattern("c6"), g) == 10


# ------------------------------------------------------------- brute force

@pytest.mark.parametrize("seed", [1, 2, 3])
@pytest.mark.parametrize("name", ["triangle", "path3", "c4", "diamond", "tailed_triangle", "k4", "house", "star4"])
def test_brute_force_tuples(seed, name):
    n = 9
    s, d = er_edges(n, 22, seed=seed)
    g = oracle.build_csr(n, s, d)
    gadj = dense(g)
    p = named_pattern(name)
    maps = brute_force_maps(p, gadj)
    assert oracle.count_maps(p, g) == maps
    assert oracle.count(p, g) * brute_force_aut(p) == maps


@pytest.mark.parametrize("seed", [4, 5])
@pytest.mark.parametrize("name", ["c5", "c6chord", "grid3x2", "k6e"])
def test_brute_force_tuples_larger_patterns(seed, name):
    n = 8
    s, d = er_edges(n, 24, seed=seed)
    g = oracle.build_csr(n, s, d)
    p = named_pattern(name)
    assert oracle.count_maps(p, g) == brute_force_maps(p, dense(g))


def test_triangles_trace_identity():
    # unordered triangles = trace(A^3) / 6
    for seed in (1, 2):
        n = 40
        s, d = er_edges(n, 300, seed=seed)
        g = oracle.build_csr(n, s, d)
        A = dense(g).astype(np.int64)
        assert oracle.triangles(g) == int(np.trace(A @ A @ A)) // 6
        assert oracle.count(named_pattern("triangle"), g) == oracle.triangles(g)


def test_root_sampling_partitions_the_maps():
    n = 60
    s, d = er_edges(n, 500, seed=9)
    g = oracle.build_csr(n, s, d)
    p = named_pattern("house")
    full = oracle.count_maps(p, g)
    parts = sum(oracle.count_maps(p, g, root_begin=r, root_stride=3) for r in range(3))
    assert parts == full


# ------------------------------------------------------ Algorithm 1 pins

def test_no_conflict_paper_example():
    # Section IV-A: after restrictions id(B) > id(D) and id(A) > id(C), the
    # permutation that sends embedding (x1,x2,x3,x4) to (x4,x1,x2,x3) is
    # eliminated (it would force x2 > x4 and x4 > x2).
    A, B, C, D = 0, 1, 2, 3
    rot = (D, A, B, C)          # rot[v]: image of v; id'(v) = id(rot[v])
    assert not pr.no_conflict(rot, {(B, D), (A, C)})
    assert pr.no_conflict((0, 1, 2, 3), {(B, D), (A, C)})     # identity survives
    assert not pr.no_conflict((0, 3, 2, 1), {(B, D)})          # (B,D) swap eliminated


@pytest.mark.parametrize("name", ["triangle", "c4", "house", "diamond", "k4", "tailed_triangle", "c5"])
def test_restriction_sets_validate_and_count(name):
    p = named_pattern(name)
    adj = p.tolist()
    k = len(adj)
    aut = len(pr.automorphisms(adj))
    sets = pr.restriction_sets(adj)
    assert sets
    n = 30
    s, d = er_edges(n, 160, seed=11)
    g = oracle.build_csr(n, s, d)
    unrestricted = oracle.count_maps(p, g)
    scheds, _ = pr.efficient_schedules(adj)
    for i, rs in enumerate(sets):
        # validate on K_k: exactly k!/|Aut| orderings survive
        assert pr.linear_extensions(k, rs) * aut == math.factorial(k)
        # the defining property on a real graph, across schedules
        sched = scheds[(7 * i) % len(scheds)]
        assert oracle.count_restricted(p, sched, rs, g) * aut == unrestricted


def test_restriction_sets_triangle_are_total_orders():
    sets = pr.restriction_sets(named_pattern("triangle").tolist())
    # every set must admit exactly one of the 3! orderings
    for rs in sets:
        assert pr.linear_extensions(3, rs) == 1
    # both orientations of every chain appear
    assert len(sets) == len({tuple(sorted((b, a) for a, b in rs)) for rs in sets})


def test_single_restriction_pattern():
    # A pattern whose only symmetry is one 2-cycle gets exactly the two
    # orientations of that pair.
    house = named_pattern("house").tolist()
    auts = pr.automorphisms(house)
    assert sorted(auts) == [(0, 1, 2, 3, 4), (1, 0, 3, 2, 4)]
    sets = pr.restriction_sets(house)
    assert sets == [((0, 1),), ((1, 0),), ((2, 3),), ((3, 2),)]


# --------------------------------------------------------------- schedules

def test_phase1_rejects_disconnected_prefix():
    # Section IV-B: searching two adjacent vertices and then a vertex adjacent
    # to neither is rejected. House: 0-1 adjacent, 4 touches only 2 and 3.
    house = named_pattern("house").tolist()
    assert not pr.phase1_ok(house, (0, 1, 4, 2, 3))
    assert pr.phase1_ok(house, (0, 1, 2, 3, 4))


def test_house_phase2_keeps_two_independent_innermost():
    house = named_pattern("house").tolist()
    assert pr.max_independent_set_size(house) == 2
    scheds, kk = pr.efficient_schedules(house)
    assert kk == 2 and scheds
    for s in scheds:
        assert not house[s[-1]][s[-2]]


def test_c4_phase1_count_and_relaxation():
    c4 = named_pattern("c4").tolist()
    p1 = [s for s in itertools.permutations(range(4)) if pr.phase1_ok(c4, s)]
    assert len(p1) == 4 * 2 * 2
    scheds, kk = pr.efficient_schedules(c4)
    # k = 2 ({0,2} or {1,3}) is infeasible: the first two would be non-adjacent
    assert pr.max_independent_set_size(c4) == 2 and kk == 1 and len(scheds) == 16


# ---------------------------------------------------------- performance model

def test_f_single_restriction_is_half():
    # Section IV-C: id(A) > id(B) filters half of the n! relative orders.
    f = pr.f_values(5, (0, 1, 2, 3, 4), [(0, 1)])
    assert f[1] == 0.5 and sum(f) == 0.5


@pytest.mark.parametrize("name", ["triangle", "house", "k4", "c5", "diamond"])
def test_f_survivors_equal_one_over_aut(name):
    adj = named_pattern(name).tolist()
    k = len(adj)
    aut = len(pr.automorphisms(adj))
    scheds, _ = pr.efficient_schedules(adj)
    for rs in pr.restriction_sets(adj)[:8]:
        for s in scheds[:5]:
            surv = 1.0
            for f in pr.f_values(k, s, rs):
                surv *= 1.0 - f
            assert abs(surv - 1.0 / aut) < 1e-12


def test_cardinality_estimates_match_graph_means():
    # |N| estimate 2|E|/|V| is the mean degree; the 2-way estimate
    # |V| p1 p2 is the mean common-neighbour count of a directed edge when
    # tri_cnt counts ordered triangles.
    n = 200
    s, d = er_edges(n, 2500, seed=3)
    g = oracle.build_csr(n, s, d)
    A = dense(g).astype(np.int64)
    E = g.nnz // 2
    T = oracle.triangles(g)
    p1, p2 = pr.graph_params(n, E, 6 * T)
    assert abs(n * p1 - A.sum(axis=1).mean()) < 1e-9
    common = (A @ A)[A == 1]
    assert abs(n * p1 * p2 - common.mean()) < 1e-9


def test_listing_is_the_set_of_embeddings():
    # every listed tuple is an edge-preserving injective map obeying the
    # restrictions, they are pairwise distinct, and there are count(P, G)
    # of them; brute force gives the same set
    n = 9
    s, d = er_edges(n, 22, seed=3)
    g = oracle.build_csr(n, s, d)
    gadj = dense(g)
    for name in ("house", "c4", "diamond", "path4"):
        p = named_pattern(name)
        adj = p.tolist()
        k = len(adj)
        sched = pr.efficient_schedules(adj)[0][0]
        rs = pr.restriction_sets(adj)[0]
        tuples, total = oracle.list_restricted(p, sched, rs, g)
        assert total == len(tuples) == oracle.count(p, g)
        got = {tuple(t) for t in tuples}
        assert len(got) == total
        pe = [(a, b) for a in range(k) for b in range(k) if adj[a][b]]
        brute = {t for t in itertools.permutations(range(n), k)
                 if all(gadj[t[a], t[b]] for a, b in pe) and all(t[a] > t[b] for a, b in rs)}
        assert got == brute


# ------------------------------------------------------------ labelled pins

def test_labeled_uniform_labels_reduce_to_unlabeled():
    n = 40
    s, d = er_edges(n, 300, seed=8)
    g = oracle.build_csr(n, s, d)
    for name in ("house", "c4", "diamond"):
        p = named_pattern(name)
        k = p.shape[0]
        assert oracle.count_labeled(p, [7] * k, g, [7] * n) == oracle.count(p, g)
        assert oracle.aut_count_labeled(p, [7] * k) == oracle.aut_count(p)


def test_labeled_alternating_cycle_in_bipartite():
    # K_{a,b} with the two sides labelled 0 and 1: every 4-cycle alternates,
    # so the 4-cycle labelled 0,1,0,1 has C(a,2) C(b,2) embeddings and the
    # labelling 0,0,1,1 has none
    for a, b in ((3, 4), (4, 5)):
        g = bipartite(a, b)
        gl = [0] * a + [1] * b
        c4 = named_pattern("c4")
        assert oracle.count_labeled(c4, [0, 1, 0, 1], g, gl) == math.comb(a, 2) * math.comb(b, 2)
        assert oracle.count_labeled(c4, [0, 0, 1, 1], g, gl) == 0
        assert oracle.aut_count_labeled(c4, [0, 1, 0, 1]) == 4


@pytest.mark.parametrize("seed", [1, 2])
def test_labeled_brute_force(seed):
    n = 9
    s, d = er_edges(n, 24, seed=seed)
    g = oracle.build_csr(n, s, d)
    gadj = dense(g)
    gl = [(7 * v + seed) % 3 for v in range(n)]
    for name, pl in (("triangle", [0, 1, 1]), ("house", [0, 0, 1, 2, 1]), ("path4", [2, 0, 0, 1])):
        p = named_pattern(name)
        k = p.shape[0]
        pe = [(x, y) for x in range(k) for y in range(k) if p[x, y]]
        maps = sum(1 for t in itertools.permutations(range(n), k)
                   if all(gadj[t[x], t[y]] for x, y in pe) and all(gl[t[x]] == pl[x] for x in range(k)))
        aut = sum(1 for q in itertools.permutations(range(k))
                  if all(p[q[x], q[y]] for x, y in pe) and all(pl[q[x]] == pl[x] for x in range(k)))
        assert oracle.aut_count_labeled(p, pl) == aut
        assert oracle.count_labeled(p, pl, g, gl) == maps // aut


def test_entry_ranges_partition_the_restricted_count():
    """The restricted count over CSR entry ranges: a root's row gives the
    root's count, and any cut of all entries adds up to the whole count."""
    for seed, pname in [(3, "house"), (4, "k4"), (5, "c5"), (6, "diamond")]:
        s, d = er_edges(40, 260, seed=seed)
        g = oracle.build_csr(40, s, d)
        adj = named_pattern(pname)
        sched = pr.efficient_schedules(adj.tolist())[0][0]
        rs = pr.restriction_sets(adj.tolist())[-1]
        whole = oracle.count_restricted(adj, sched, rs, g)
        nnz = int(g.row_ptr[-1])
        cuts = [0, 1, 7, nnz // 2, nnz - 3, nnz]
        assert sum(oracle.count_restricted_entries(adj, sched, rs, g, a, b) for a, b in zip(cuts, cuts[1:])) == whole
        for r in (0, 5, 39):
            assert oracle.count_restricted_entries(adj, sched, rs, g, g.row_ptr[r], g.row_ptr[r + 1]) == \
                oracle.count_restricted(adj, sched, rs, g, root_begin=r, root_end=r + 1)
