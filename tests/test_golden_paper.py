"""The paper's worked examples (tests/golden/paper_worked_examples.json,
each entry citing its section) against the oracle's restatement of the
method, plus the inclusion-exclusion count of Section IV-D against brute
force. CPU only."""

import itertools
import json
import math
import os
import random

import pytest

import oracle
from oracle import planner_ref as pr

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "paper_worked_examples.json")


def examples():
    with open(GOLDEN) as f:
        return {e["id"]: e for e in json.load(f)["examples"]}


def adj_from_edges(k, edges):
    import numpy as np
    a = np.zeros((k, k), np.uint8)
    for x, y in edges:
        a[x, y] = a[y, x] = 1
    return a


def test_every_example_cites_a_section():
    for e in examples().values():
        assert e["cite"].startswith("Section ")


def test_rectangle_b_d_swap():
    e = examples()["rectangle_b_d_swap"]
    adj = adj_from_edges(4, e["pattern_edges"])
    auts = pr.automorphisms(adj.tolist())
    assert tuple(e["automorphism"]) in auts
    assert oracle.aut_count(adj) == len(auts) == 8


def test_no_conflict_round_one():
    e = examples()["no_conflict_round_one"]
    res = {tuple(r) for r in e["restrictions"]}
    assert pr.no_conflict(tuple(e["permutation"]), res) is (not e["eliminated"])


def test_f_one_half():
    e = examples()["f_one_half"]
    assert math.factorial(e["n"]) == e["relative_orders"]
    assert pr.f_values(e["n"], tuple(e["schedule"]), [tuple(r) for r in e["restrictions"]]) == e["f"]


def test_algorithm2_components():
    e = examples()["algorithm2_components"]
    pairs = [tuple(p) for p in e["pairs"]]
    assert pr.components(e["k"], pairs) == e["components"]
    # |A12 ∩ A23 ∩ A45| = |S1 ∩ S2 ∩ S3| x |S4 ∩ S5| x |S6|
    rng = random.Random(7)
    sets = [set(rng.sample(range(12), rng.randint(3, 9))) for _ in range(e["k"])]
    expect = len(sets[0] & sets[1] & sets[2]) * len(sets[3] & sets[4]) * len(sets[5])
    assert pr.intersection_card(e["k"], pairs, sets) == expect
    brute = sum(1 for t in itertools.product(*sets) if t[0] == t[1] == t[2] and t[3] == t[4])
    assert brute == expect


@pytest.mark.parametrize("k", [2, 3, 4])
def test_iep_count_equals_distinct_tuples(k):
    rng = random.Random(k)
    for _ in range(20):
        sets = [set(rng.sample(range(9), rng.randint(0, 7))) for _ in range(k)]
        brute = sum(1 for t in itertools.product(*sets) if len(set(t)) == k)
        assert pr.iep_count(sets) == brute
        if k == 2:          # the form the count kernel evaluates
            assert brute == len(sets[0]) * len(sets[1]) - len(sets[0] & sets[1])


def test_k7_automorphisms():
    e = examples()["k7_automorphisms"]
    adj = adj_from_edges(e["k"], [(a, b) for a in range(e["k"]) for b in range(a + 1, e["k"])])
    assert oracle.aut_count(adj) == len(pr.automorphisms(adj.tolist())) == e["automorphisms"]


def test_house_phase2():
    e = examples()["house_phase2"]
    adj = adj_from_edges(5, e["pattern_edges"]).tolist()
    scheds, kp = pr.efficient_schedules(adj)
    assert kp == e["phase2_k"] and scheds
    assert all(not adj[s[-1]][s[-2]] for s in scheds)


@pytest.mark.parametrize("V,E,T", [(1000.0, 5000.0, 12000.0), (2.0 ** 20, 8.0 * 2 ** 20, 6.0e9)])
def test_cardinality_estimates(V, E, T):
    examples()["cardinality_estimates"]
    p1, p2 = pr.graph_params(V, E, T)
    assert math.isclose(V * p1, 2.0 * E / V, rel_tol=1e-12)             # one neighbourhood
    assert math.isclose(V * p1 * p2, T / (2.0 * E), rel_tol=1e-12)      # two adjacent vertices' lists
