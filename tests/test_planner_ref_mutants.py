"""The pins of the oracle's planner restatement (``oracle/planner_ref.py``)
catch plausible mistakes: each test swaps one function for a mutant with a
planted mistake and checks that a battery of checks fixed by the paper's
examples, by brute force or by the count invariant fails, while it passes
with the real functions. CPU only."""

import itertools
from math import factorial

import numpy as np
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
