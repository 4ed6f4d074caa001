"""Host-side check of the inclusion-exclusion divisor (no GPU): the exact
multiplicity of embeddings under the outer restrictions, counted over all
k! relative orders, against the paper's no_conflict count. Where the two
differ the exact one is right, shown by brute force on a small graph with
the oracle's restricted enumerator."""

from itertools import permutations

import oracle
from oracle import planner_ref as pr
from synth import er_edges, named_pattern


def outer(rs, sched, k):
    pos = {v: i for i, v in enumerate(sched)}
    return [(a, b) for a, b in rs if max(pos[a], pos[b]) <= k - 3]


def multiplicities(adj, ro):
    k = len(adj)
    auts = pr.automorphisms(adj)
    return {sum(1 for sg in auts if all(pi[sg[a]] > pi[sg[b]] for a, b in ro)) for pi in permutations(range(k))}


def test_grid_configuration_where_paper_divisor_differs():
    adj = named_pattern("grid3x2").tolist()
    k = len(adj)
    auts = pr.automorphisms(adj)
    scheds, _ = pr.efficient_schedules(adj)
    n = 40
    s, d = er_edges(n, 300, seed=2)
    g = oracle.build_csr(n, s, d)
    truth = oracle.count(named_pattern("grid3x2"), g)
    found = False
    for sc in scheds:
        if adj[sc[-1]][sc[-2]]:
            continue
        for rs in pr.restriction_sets(adj):
            ro = outer(rs, sc, k)
            x = sum(1 for p in auts if pr.no_conflict(p, set(ro)))
            m = multiplicities(adj, ro)
            if len(m) == 1 and x != next(iter(m)):
                # the enumeration without inner restrictions counts each
                # embedding m times, not x times
                full = oracle.count_restricted(named_pattern("grid3x2"), sc, ro, g)
                assert full == truth * next(iter(m))
                assert full != truth * x or truth == 0
                found = True
                break
        if found:
            break
    assert found
