"""CPU-side checks of the library: every symbol the header declares is
exported, and the host planner (automorphisms, Algorithm 1, schedules,
performance model) agrees exactly with the oracle's restatement."""

import os
import re

import numpy as np
import pytest

import oracle
from oracle import planner_ref as pr
from synth import er_edges, named_pattern, random_pattern_set

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def N():
    from paper_2009_10955_gb300 import native
    return native()


def declared_functions():
    text = open(os.path.join(ROOT, "include", "graphpi.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(gp_[a-z_0-9]+)\s*\(", text)))


def test_library_exports_every_declared_symbol(N):
    names = declared_functions()
    assert len(names) >= 20
    lib = N.lib()
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) == set(N.SIGNATURES)


PATTERNS = ["triangle", "c4", "house", "k4", "c5", "diamond", "k6e", "c6chord", "grid3x2",
            "tailed_triangle", "path4", "star4", "star5", "c6"]


@pytest.mark.parametrize("name", PATTERNS)
def test_planner_matches_oracle(N, name):
    adj = named_pattern(name)
    p = N.gp_pattern_create(adj)
    assert p.aut_count() == len(pr.automorphisms(adj.tolist()))
    assert set(p.restriction_sets()) == set(pr.restriction_sets(adj.tolist()))
    sc, kp = p.schedules()
    rsc, rkp = pr.efficient_schedules(adj.tolist())
    assert sc == list(rsc) and kp == rkp


def test_restriction_set_cap_and_mirrors(N):
    """A capped search returns its sets plus their mirror images (every
    restriction reversed), all valid; caps are cached side by side and the
    default cap's sets do not change after a capped call."""
    from math import factorial
    adj = named_pattern("k5")
    al = adj.tolist()
    p = N.gp_pattern_create(adj)
    full = p.restriction_sets()
    small = p.restriction_sets(cap=8)
    assert 8 <= len(small) <= 16 and len(full) == 2048
    aut = len(pr.automorphisms(al))
    for rs in small:
        assert pr.validate(5, aut, set(rs))
        assert tuple(sorted((b, a) for a, b in rs)) in {tuple(sorted(x)) for x in small}
    assert p.restriction_sets() == full and p.restriction_sets(cap=8) == small
    assert all(pr.linear_extensions(5, set(rs)) * aut == factorial(5) for rs in full[:64])


@pytest.mark.parametrize("name", ["triangle", "house", "k4", "c5", "k6e", "grid3x2"])
def test_cost_model_matches_oracle(N, name):
    adj = named_pattern(name)
    p = N.gp_pattern_create(adj)
    sets = pr.restriction_sets(adj.tolist())
    scheds, _ = pr.efficient_schedules(adj.tolist())
    for V, E, T in [(2000.0, 19905.0, 6 * 1301.0), (1048576.0, 15700364.0, 6.0e9), (10.0, 20.0, 0.0)]:
        for s in scheds[:12]:
            for r in sets[:12]:
                a = N.gp_config_cost(p, s, r, V, E, T)
                b = pr.cost(adj.tolist(), s, r, V, E, T)
                assert abs(a - b) <= 1e-12 * max(abs(b), 1e-300)


def test_random_patterns_planner(N):
    for adj in random_pattern_set(12, 3, 5, 0.5, seed=5):
        p = N.gp_pattern_create(adj)
        assert set(p.restriction_sets()) == set(pr.restriction_sets(adj.tolist()))
        assert p.schedules()[0] == list(pr.efficient_schedules(adj.tolist())[0])


def test_schedule_top_k_is_sorted_by_cost(N):
    p = N.gp_pattern_create(named_pattern("house"))
    s = N.gp_schedule(p, None, top_k=5)
    costs = [s.get(i)[2] for i in range(len(s))]
    assert costs == sorted(costs)
    rows = pr.all_configurations(named_pattern("house").tolist(), float(1 << 20), 8.0 * (1 << 20),
                                 6.0 * 8.0 * (1 << 20))
    assert abs(costs[0] - rows[0][0]) <= 1e-12 * rows[0][0]


def test_bad_patterns_rejected(N):
    bad = [np.zeros((2, 2), np.uint8),                      # too small
           np.zeros((8, 8), np.uint8),                      # too large
           np.array([[0, 1, 0], [0, 0, 1], [0, 1, 0]], np.uint8),   # asymmetric
           np.array([[1, 1, 0], [1, 0, 1], [0, 1, 0]], np.uint8),   # self loop
           np.array([[0, 1, 0, 0], [1, 0, 0, 0], [0, 0, 0, 1], [0, 0, 1, 0]], np.uint8)]  # disconnected
    for adj in bad:
        with pytest.raises(N.GraphPiError) as e:
            N.gp_pattern_create(adj)
        assert e.value.status == N.GP_ERR_PATTERN


def test_explicit_schedule_validation(N):
    p = N.gp_pattern_create(named_pattern("triangle"))
    with pytest.raises(N.GraphPiError):
        N.gp_schedule_explicit(p, (0, 1, 2), [(0, 1)])         # leaves 3 of 6 orders: invalid
    N.gp_schedule_explicit(p, (0, 1, 2), [(0, 1), (1, 2)])
    c4 = N.gp_pattern_create(named_pattern("c4"))
    with pytest.raises(N.GraphPiError):
        N.gp_schedule_explicit(c4, (0, 2, 1, 3), [(0, 1), (0, 2), (1, 3)])  # disconnected prefix


@pytest.mark.parametrize("name,labels", [("house", [0, 0, 1, 1, 2]), ("house", [0, 1, 0, 1, 2]),
                                         ("c4", [0, 1, 0, 1]), ("k4", [0, 0, 1, 1]), ("diamond", [1, 1, 0, 0])])
def test_labeled_planner_matches_oracle(N, name, labels):
    import oracle
    adj = named_pattern(name)
    p = N.gp_pattern_create_labeled(adj, labels)
    assert p.aut_count() == len(pr.automorphisms(adj.tolist(), labels)) == oracle.aut_count_labeled(adj, labels)
    assert set(p.restriction_sets()) == set(pr.restriction_sets(adj.tolist(), labels))


def test_status_strings_cover_every_code(N):
    lib = N.lib()
    seen = set()
    for code in (0, 1, -1, -2, -3, -4, -5, -6, -7, -8):
        s = lib.gp_status_str(code).decode()
        assert s and s not in seen, code
        seen.add(s)
    assert lib.gp_status_str(-99).decode()                 # unknown codes still get a string


def test_host_calls_reject_bad_arguments(N):
    import ctypes
    lib = N.lib()
    out = ctypes.c_void_p()
    adj = np.ascontiguousarray(named_pattern("house"), dtype=np.uint8)
    assert lib.gp_pattern_create(None, 5, ctypes.byref(out)) == N.GP_ERR_ARG
    assert lib.gp_pattern_create(adj.ctypes.data_as(ctypes.c_void_p), 5, None) == N.GP_ERR_ARG
    assert lib.gp_pattern_create_labeled(adj.ctypes.data_as(ctypes.c_void_p), None, 5,
                                         ctypes.byref(out)) == N.GP_ERR_ARG
    assert lib.gp_last_error().decode()                    # the failure left a message
    p = N.gp_pattern_create(adj)
    s = N.gp_schedule(p, None, top_k=2)
    order = (ctypes.c_int32 * 7)()
    assert lib.gp_schedule_get(s.h, 5, order, None, None, None) == N.GP_ERR_ARG   # idx out of range
    assert lib.gp_schedule_get(s.h, -1, order, None, None, None) == N.GP_ERR_ARG
    cnt = ctypes.c_int32()
    assert lib.gp_schedule_size(s.h, ctypes.byref(cnt)) == N.GP_OK and cnt.value == 2
    assert lib.gp_schedule(p.h, None, 0, None, ctypes.byref(out)) == N.GP_ERR_ARG   # top_k >= 1


def test_iep_switch_on_plans_that_do_not_qualify(N):
    import ctypes
    lib = N.lib()
    n_iep = ctypes.c_int32(-1)
    tri = N.gp_schedule(N.gp_pattern_create(named_pattern("triangle")), None)
    assert lib.gp_schedule_set_iep(tri.h, 1, ctypes.byref(n_iep)) == N.GP_OK and n_iep.value == 0
    k4 = N.gp_schedule(N.gp_pattern_create(named_pattern("k4")), None)        # last two adjacent
    assert lib.gp_schedule_set_iep(k4.h, 1, ctypes.byref(n_iep)) == N.GP_OK and n_iep.value == 0
    house = N.gp_schedule(N.gp_pattern_create(named_pattern("house")), None, top_k=3)
    assert lib.gp_schedule_set_iep(house.h, 1, ctypes.byref(n_iep)) == N.GP_OK and n_iep.value >= 1
    assert lib.gp_schedule_set_iep(house.h, 0, ctypes.byref(n_iep)) == N.GP_OK


def _iep_form(adj, order, res):
    """The innermost-loop count kk and divisor that the definitions of
    Section IV-D give for one configuration: the largest kk <= min(k - 2, 5)
    whose last kk vertices are pairwise non-adjacent and for which the
    number of automorphic copies obeying the outer restrictions is the same
    for every relative order of the k vertices."""
    from itertools import permutations
    k = len(adj)
    auts = pr.automorphisms(adj)
    pos = {v: i for i, v in enumerate(order)}
    for kk in range(min(k - 2, 5), 1, -1):
        inner = order[k - kk:]
        if any(adj[a][b] for a in inner for b in inner if a != b):
            continue
        ro = [(a, b) for a, b in res if max(pos[a], pos[b]) < k - kk]
        m = {sum(1 for sg in auts if all(pi[sg[a]] > pi[sg[b]] for a, b in ro)) for pi in permutations(range(k))}
        if len(m) == 1 and next(iter(m)) > 0:
            return kk, next(iter(m))
    return 0, 1


@pytest.mark.parametrize("name", ["house", "k6e", "c6chord", "grid3x2", "star4", "star5", "star6", "star7",
                                  "three_ears", "path5", "k4"])
def test_iep_form_of_top_plans(N, name):
    adj = named_pattern(name)
    sc = N.gp_schedule(N.gp_pattern_create(adj), None, top_k=4)
    sc.set_iep(True)
    for i in range(len(sc)):
        order, res, _ = sc.get(i)
        assert sc.iep(i) == _iep_form(adj.tolist(), list(order), list(res)), (name, i, order, res)
    sc.set_iep(False)
    assert all(sc.iep(i) == (0, 1) for i in range(len(sc)))


@pytest.mark.parametrize("name", ["c5", "house", "diamond", "tailed_triangle", "three_ears", "star5",
                                  "path5", "grid3x2", "c6chord"])
def test_iep_form_of_every_configuration(N, name):
    """Sampled configurations (efficient schedule x Algorithm 1 set), not
    only the model's top plans: the planner's kk and divisor equal the
    definition's; a 5-cycle has no configuration with an inclusion-exclusion
    form (every order with connected prefixes ends in an adjacent pair)."""
    adj = named_pattern(name)
    p = N.gp_pattern_create(adj)
    scheds, _ = p.schedules()
    sets = p.restriction_sets()
    pairs = [(s, r) for s in scheds for r in sets]
    step = max(1, len(pairs) // 60)
    forms = []
    for s, r in pairs[::step]:
        sc = N.gp_schedule_explicit(p, s, r)
        sc.set_iep(True)
        forms.append(sc.iep(0))
        assert forms[-1] == _iep_form(adj.tolist(), list(s), [tuple(x) for x in r]), (name, s, r)
    if name == "c5":
        assert all(f == (0, 1) for f in forms)
    else:
        assert any(f[0] >= 2 for f in forms)


def test_labeled_pattern_groups(N):
    # equal labels give the plain group; alternating labels keep the
    # rotations by two and the reflections that fix the label classes;
    # distinct labels leave the identity
    adj = named_pattern("c4")
    p = N.gp_pattern_create_labeled(adj, [3, 3, 3, 3])
    assert p.aut_count() == N.gp_pattern_create(adj).aut_count() == 8
    assert N.gp_pattern_create_labeled(adj, [0, 1, 0, 1]).aut_count() == 4
    assert N.gp_pattern_create_labeled(adj, [0, 1, 2, 3]).aut_count() == 1


def test_directed_patterns_host_side(N):
    """Directed patterns (host): arc-preserving groups against the oracle's,
    and malformed matrices rejected."""
    import oracle

    def pat(k, arcs):
        a = np.zeros((k, k), np.uint8)
        for x, y in arcs:
            a[x, y] = 1
        return a
    cases = [pat(3, [(0, 1), (1, 2), (2, 0)]), pat(3, [(0, 1), (0, 2), (1, 2)]),
             pat(4, [(0, 1), (1, 2), (2, 3), (3, 0)]), pat(4, [(0, 2), (0, 3), (1, 2), (1, 3)]),
             pat(4, [(0, 1), (0, 2), (0, 3)]), pat(3, [(0, 1), (1, 0), (0, 2), (1, 2)])]
    for a in cases:
        assert N.gp_dpattern_create(a).aut_count() == oracle.aut_count_directed(a)
    for bad in (pat(3, [(0, 1)]),                              # not weakly connected
                pat(2, [(0, 1)]),                              # too small
                np.eye(3, dtype=np.uint8)):                    # loops
        with pytest.raises(N.GraphPiError) as e:
            N.gp_dpattern_create(bad)
        assert e.value.status == N.GP_ERR_PATTERN


def test_plan_candidates_are_top_plans_and_mirrors(N):
    """autotune.plan_candidates: the model's top plans in rank order, each
    followed by its mirror image (every restriction reversed, a valid set of
    the same model cost), no repeats."""
    from paper_2009_10955_gb300 import autotune
    for name in ("house", "k4", "k6e", "three_ears"):
        adj = named_pattern(name)
        p = N.gp_pattern_create(adj)
        top = N.gp_schedule(p, None, top_k=3)
        cands = autotune.plan_candidates(p, None, top_k=3)
        assert len(set(cands)) == len(cands)
        assert cands[0] == (top.get(0)[0], tuple(top.get(0)[1]))
        aut = len(pr.automorphisms(adj.tolist()))
        firsts = [(top.get(i)[0], tuple(top.get(i)[1])) for i in range(len(top))]
        for order, res in cands:
            mirror = tuple((b, a) for a, b in res)
            assert (order, res) in firsts or (order, mirror) in firsts
            assert pr.validate(len(adj), aut, set(res))
            c = N.gp_config_cost(p, order, res, 2.0 ** 20, 8.0 * 2 ** 20, 6.0 * 8 * 2 ** 20)
            m = N.gp_config_cost(p, order, mirror, 2.0 ** 20, 8.0 * 2 ** 20, 6.0 * 8 * 2 ** 20)
            assert abs(c - m) <= 1e-12 * c


@pytest.mark.parametrize("name", ["c7", "k7", "star7"])
def test_seven_vertex_sets_are_valid(N, name):
    """7-vertex patterns, whose full restriction-set search the oracle's
    restatement cannot finish quickly: every library set passes validate
    (Section IV-A), mirror images come in pairs, and on a small graph a
    sample of the sets times |Aut| gives the unrestricted map count."""
    adj = named_pattern(name)
    al = adj.tolist()
    p = N.gp_pattern_create(adj)
    aut = len(pr.automorphisms(al))
    assert p.aut_count() == aut
    sets = p.restriction_sets()
    keyed = {tuple(sorted(r)) for r in sets}
    for r in sets:
        assert pr.validate(7, aut, set(r))
        assert tuple(sorted((b, a) for a, b in r)) in keyed
    s, d = er_edges(14, 60, seed=3)
    g = oracle.build_csr(14, s, d)
    maps = oracle.count_maps(adj, g)
    sched = p.schedules()[0][0]
    for r in sets[:: max(1, len(sets) // 6)]:
        assert oracle.count_restricted(adj, sched, r, g) * aut == maps, r
