"""Closed forms of the performance model (Section IV-C) for schedules whose
terms can be written out by hand, pinning the recursion that combines l_i,
f_i and c_i: cost_i = l_i (1 - f_i) (c_i + cost_{i+1}), cost_n = l_n (1 - f_n),
with |N| = |V| p1 for a neighbourhood and |V| p1 p2^(m-1) for an m-way
intersection (p1 = 2|E|/|V|^2, p2 = tri_cnt |V| / (2|E|)^2). CPU only."""

import numpy as np
import pytest

from oracle import planner_ref as pr
from synth import named_pattern

GRAPHS = [(1000.0, 5000.0, 6.0 * 2000.0), (2.0 ** 20, 8.0 * 2.0 ** 20, 6.0 * 3.0e7), (50.0, 300.0, 0.0)]


def params(V, E, T):
    return 2.0 * E / (V * V), T * V / (2.0 * E) ** 2


def close(a, b):
    return abs(a - b) <= 1e-12 * max(abs(b), 1e-300)


def edges_adj(k, edges):
    a = np.zeros((k, k), np.uint8)
    for x, y in edges:
        a[x, y] = a[y, x] = 1
    return a.tolist()


@pytest.mark.parametrize("V,E,T", GRAPHS)
def test_intersection_free_schedules(V, E, T):
    # a path or a star searched from one end / the centre: every later vertex
    # iterates one neighbourhood (l = |V| p1), nothing is intersected (c = 0)
    # and nothing is restricted (f = 0), so cost = |V| (|V| p1)^(k-1)
    p1, _ = params(V, E, T)
    for k in (3, 4, 5):
        path = edges_adj(k, [(i, i + 1) for i in range(k - 1)])
        star = edges_adj(k, [(0, i) for i in range(1, k)])
        for adj in (path, star):
            assert close(pr.cost(adj, tuple(range(k)), (), V, E, T), V * (V * p1) ** (k - 1))


@pytest.mark.parametrize("V,E,T", GRAPHS)
def test_triangle_with_and_without_restrictions(V, E, T):
    p1, p2 = params(V, E, T)
    tri = named_pattern("triangle").tolist()
    n1, n2 = V * p1, V * p1 * p2           # a neighbourhood, a 2-way intersection
    # loop 2 builds N(v0) ∩ N(v1) from two neighbourhood-sized operands
    plain = V * (n1 * (2 * n1 + n2))
    assert close(pr.cost(tri, (0, 1, 2), (), V, E, T), plain)
    # id(0) > id(1) removes half of the orders at loop 2, id(1) > id(2) two
    # thirds of the rest at loop 3
    restricted = V * (n1 * 0.5 * (2 * n1 + n2 * (1.0 / 3.0)))
    assert close(pr.cost(tri, (0, 1, 2), ((0, 1), (1, 2)), V, E, T), restricted)


@pytest.mark.parametrize("V,E,T", GRAPHS)
def test_four_cycle_shares_no_intersection_until_the_last_vertex(V, E, T):
    # C4 searched 0, 1, 3, 2 (edges 0-1, 1-2, 2-3, 3-0): vertex 1 and vertex 3
    # iterate N(v0); vertex 2 iterates N(v1) ∩ N(v3), built at loop 3 from
    # N(v1) and N(v3); no restrictions
    p1, p2 = params(V, E, T)
    c4 = named_pattern("c4").tolist()
    n1, n2 = V * p1, V * p1 * p2
    expect = V * (n1 * (n1 * (2 * n1 + n2)))
    assert close(pr.cost(c4, (0, 1, 3, 2), (), V, E, T), expect)
