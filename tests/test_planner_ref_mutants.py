"""The pins of the oracle's planner restatement (``oracle/planner_ref.py``)
catch plausible mistakes: each test swaps one function for a mutant with a
planted mistake and checks that a battery of checks fixed by the paper's
examples, by brute force or by the count invariant fails, while it passes
with the real functions. CPU only."""

import itertools
from math import factorial

import pytest

import oracle
from oracle import planner_ref as pr
from synth import er_edges, named_pattern


def brute_schedules(adj):
    """Section IV-B by brute force: connected prefixes, then the largest
    k' <= k whose last k' vertices are pairwise non-adjacent in some schedule."""
    k = len(adj)

    def connected_prefixes(s):
        return all(any(adj[s[i]][s[j]] for j in range(i)) for i in range(1, k))

    p1 = [s for s in itertools.permutations(range(k)) if connected_prefixes(s)]
    for kk in range(k, 0, -1):
        out = [s for s in p1 if all(not adj[a][b] for a, b in itertools.combinations(s[k - kk:], 2))]
        if out:
            return out, kk
    return p1, 1


def battery():
    failed = []

    def check(name, ok):
        if not ok:
            failed.append(name)
    try:
        c4 = named_pattern("c4").tolist()
        auts = pr.automorphisms(c4)
        check("rectangle_group", len(auts) == 8 and (0, 3, 2, 1) in auts)
        A, B, C, D = 0, 1, 2, 3
        check("no_conflict_example", not pr.no_conflict((D, A, B, C), {(B, D), (A, C)})
              and pr.no_conflict((0, 1, 2, 3), {(B, D), (A, C)}))
        s, d = er_edges(30, 140, seed=2)
        g = oracle.build_csr(30, s, d)
        for name in ("triangle", "c4", "house", "diamond", "path5"):
            adj = named_pattern(name)
            al = adj.tolist()
            aut = len(pr.automorphisms(al))
            sets = pr.restriction_sets(al)
            check(f"{name}_has_sets", len(sets) > 0)
            maps = oracle.count_maps(adj, g)
            sched = brute_schedules(al)[0][0]
            for rs in sets[:4]:
                check(f"{name}_count_invariant", oracle.count_restricted(adj, sched, rs, g) * aut == maps)
                f = pr.f_values(len(al), sched, rs)
                prod = 1.0
                for x in f:
                    prod *= 1.0 - x
                check(f"{name}_f_product", abs(prod - 1.0 / aut) < 1e-12)
            check(f"{name}_schedules", [tuple(x) for x in pr.efficient_schedules(al)[0]] == brute_schedules(al)[0]
                  and pr.efficient_schedules(al)[1] == brute_schedules(al)[1])
        check("f_one_half", pr.f_values(5, (0, 1, 2, 3, 4), [(0, 1)])[1] == 0.5)
    except Exception as e:
        failed.append(f"raised {type(e).__name__}")
    return failed


def m_no_conflict_ignores_perm(perm, res_set):
    return pr._acyclic(len(perm), list(res_set))


def m_automorphisms_drop_an_edge(adj, labels=None):
    k = len(adj)
    E = [(a, b) for a in range(k) for b in range(a + 1, k) if adj[a][b]][:-1]   # one edge unchecked
    return [p for p in itertools.permutations(range(k)) if all(adj[p[a]][p[b]] for a, b in E)]


def m_validate_always(k, aut_count, res_set):
    return True


def m_f_over_all_orders(k, sched, res_set):
    pos = {v: i for i, v in enumerate(sched)}
    alive = list(itertools.permutations(range(k)))
    f = []
    for i in range(k):
        here = [(a, b) for a, b in res_set if max(pos[a], pos[b]) == i]
        before = len(alive)
        for a, b in here:
            alive = [s for s in alive if s[a] > s[b]]
        f.append(0.0 if not here else (before - len(alive)) / factorial(k))
    return f


def m_phase2_consecutive_only(adj, sched, kk):
    tail = sched[len(sched) - kk:]
    return all(not adj[a][b] for a, b in zip(tail, tail[1:]))


def m_linear_extensions_reversed(k, res_set):
    return sum(1 for sigma in itertools.permutations(range(k)) if all(sigma[a] < sigma[b] for a, b in res_set)) + 1


MUTANTS = [
    ("no_conflict", m_no_conflict_ignores_perm),
    ("automorphisms", m_automorphisms_drop_an_edge),
    ("validate", m_validate_always),
    ("f_values", m_f_over_all_orders),
    ("phase2_ok", m_phase2_consecutive_only),
    ("linear_extensions", m_linear_extensions_reversed),
]


def test_real_planner_passes_the_battery():
    assert battery() == []


@pytest.mark.parametrize("fname,mutant", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planner_mutant_is_caught(monkeypatch, fname, mutant):
    monkeypatch.setattr(pr, fname, mutant)
    assert battery(), f"mutant of {fname} passed every check"


# ------------------------------------------- cost model and inclusion-exclusion
# A second battery for the performance model (Section IV-C) and the
# inclusion-exclusion functions (Section IV-D, Algorithm 2): closed forms of
# the cost written out by hand, the Algorithm 2 components example, brute
# force over distinct tuples, and whole-count agreement of the IEP total of
# an unrestricted plan with the number of injective maps.

def _edges_adj(k, edges):
    a = [[0] * k for _ in range(k)]
    for x, y in edges:
        a[x][y] = a[y][x] = 1
    return a


def model_battery():
    import random
    failed = []

    def check(name, ok):
        if not ok:
            failed.append(name)
    try:
        V, E, T = 1000.0, 5000.0, 12000.0
        p1, p2 = 2.0 * E / (V * V), T * V / (2.0 * E) ** 2
        n1, n2 = V * p1, V * p1 * p2

        def close(a, b):
            return abs(a - b) <= 1e-12 * abs(b)
        check("graph_params", all(close(x, y) for x, y in zip(pr.graph_params(V, E, T), (p1, p2))))
        path = _edges_adj(4, [(0, 1), (1, 2), (2, 3)])
        check("cost_path", close(pr.cost(path, (0, 1, 2, 3), (), V, E, T), V * n1 ** 3))
        tri = named_pattern("triangle").tolist()
        check("cost_triangle", close(pr.cost(tri, (0, 1, 2), (), V, E, T), V * n1 * (2 * n1 + n2)))
        check("cost_triangle_restricted",
              close(pr.cost(tri, (0, 1, 2), ((0, 1), (1, 2)), V, E, T), V * n1 * 0.5 * (2 * n1 + n2 / 3.0)))
        c4 = named_pattern("c4").tolist()
        check("cost_c4", close(pr.cost(c4, (0, 1, 3, 2), (), V, E, T), V * n1 * n1 * (2 * n1 + n2)))
        # Algorithm 2's partition example: pairs (1,2), (2,3), (4,5) of six sets
        pairs = [(1, 2), (2, 3), (4, 5)]
        check("components", pr.components(6, pairs) == [[1, 2, 3], [4, 5], [6]])
        rng = random.Random(3)
        sets6 = [set(rng.sample(range(12), rng.randint(3, 9))) for _ in range(6)]
        check("intersection_card", pr.intersection_card(6, pairs, sets6)
              == len(sets6[0] & sets6[1] & sets6[2]) * len(sets6[3] & sets6[4]) * len(sets6[5]))
        for k in (2, 3, 4):
            for _ in range(8):
                sets = [set(rng.sample(range(8), rng.randint(0, 6))) for _ in range(k)]
                brute = sum(1 for t in itertools.product(*sets) if len(set(t)) == k)
                check(f"iep_count_k{k}", pr.iep_count(sets) == brute)
        s, d = er_edges(24, 110, seed=4)
        g = oracle.build_csr(24, s, d)
        for name, sched, kk in (("house", (2, 3, 1, 4, 0), 2), ("star5", (0, 1, 2, 3, 4), 3)):
            adj = named_pattern(name)
            check(f"iep_total_{name}", oracle.iep_total(adj, sched, (), kk, g) == oracle.count_maps(adj, g))
    except Exception as e:
        failed.append(f"raised {type(e).__name__}")
    return failed


def m_graph_params_p2_unsquared(n_vertices, n_edges, tri_cnt):
    V, E = float(n_vertices), float(n_edges)
    return 2.0 * E / (V * V), tri_cnt * V / (2.0 * E)


def _cost_with(adj, sched, res_set, n_vertices, n_edges, tri_cnt, card_shift=0, drop_f_inner=False,
               prefix_card_shift=0):
    """The cost recursion of Section IV-C with one term shifted or dropped."""
    k = len(adj)
    V = float(n_vertices)
    p1, p2 = pr.graph_params(n_vertices, n_edges, tri_cnt)

    def card(m):
        return V if m == 0 else V * p1 * p2 ** (m - 1 + card_shift)

    ops = [[j for j in range(i) if adj[sched[i]][sched[j]]] for i in range(k)]
    l = [card(len(ops[i])) for i in range(k)]
    c = [0.0] * k
    for i in range(k):
        built = set()
        for x in range(i + 1, k):
            O = ops[x]
            if i in O and O.index(i) >= 1:
                prefix = tuple(j for j in O if j <= i)
                if prefix in built:
                    continue
                built.add(prefix)
                c[i] += card(len(prefix) - 1 + prefix_card_shift) + card(1)
    f = pr.f_values(k, sched, res_set)
    total = l[k - 1] * (1.0 - f[k - 1])
    for i in range(k - 2, -1, -1):
        total = l[i] * (1.0 if drop_f_inner else 1.0 - f[i]) * (c[i] + total)
    return total


def m_cost_card_exponent(*a):
    return _cost_with(*a, card_shift=1)


def m_cost_drops_outer_f(*a):
    return _cost_with(*a, drop_f_inner=True)


def m_cost_prefix_card(*a):
    return _cost_with(*a, prefix_card_shift=1)


def m_components_ignore_chains(k, pairs):
    # only the first pair of each vertex joins it: (2, 3) after (1, 2) is lost
    seen, comps = set(), []
    for i, j in pairs:
        if i in seen or j in seen:
            continue
        seen |= {i, j}
        comps.append([i, j])
    comps += [[v] for v in range(1, k + 1) if v not in seen]
    return sorted(comps)


def m_intersection_card_union(k, pairs, sets):
    card = 1
    for comp in pr.components(k, pairs):
        common = set()
        for v in comp:
            common |= set(sets[v - 1])
        card *= len(common)
    return card


def m_iep_count_no_sign(sets):
    k = len(sets)
    all_pairs = [(i, j) for i in range(1, k + 1) for j in range(i + 1, k + 1)]
    return sum(pr.intersection_card(k, sub, sets)
               for m in range(len(all_pairs) + 1) for sub in itertools.combinations(all_pairs, m))


def m_iep_count_pairs_only(sets):
    # stops the expansion after the single pairs (the first-order terms)
    k = len(sets)
    all_pairs = [(i, j) for i in range(1, k + 1) for j in range(i + 1, k + 1)]
    total = pr.intersection_card(k, (), sets)
    for p in all_pairs:
        total -= pr.intersection_card(k, (p,), sets)
    return total


MODEL_MUTANTS = [
    ("graph_params", m_graph_params_p2_unsquared),
    ("cost", m_cost_card_exponent),
    ("cost", m_cost_drops_outer_f),
    ("cost", m_cost_prefix_card),
    ("components", m_components_ignore_chains),
    ("intersection_card", m_intersection_card_union),
    ("iep_count", m_iep_count_no_sign),
    ("iep_count", m_iep_count_pairs_only),
]


def test_real_model_passes_the_battery():
    assert model_battery() == []


@pytest.mark.parametrize("fname,mutant", MODEL_MUTANTS, ids=[m[1].__name__[2:] for m in MODEL_MUTANTS])
def test_model_mutant_is_caught(monkeypatch, fname, mutant):
    monkeypatch.setattr(pr, fname, mutant)
    assert model_battery(), f"mutant {mutant.__name__} passed every check"
