"""Named and seeded random patterns, as k x k symmetric 0/1 uint8 matrices.

Named patterns follow the workloads the counts are quoted on:

* ``triangle``, ``k4``, ``k5``, ``k6``, ``k7`` (cliques);
* ``house``: edges 0-1, 1-2, 2-3, 3-0, 2-4, 3-4 (a square with a roof);
* ``c4`` .. ``c7``: cycles 0-1-...-(k-1)-0;
* ``k6e``: the 6-clique minus the edge 0-1;
* ``c6chord``: the 6-cycle plus the chord 0-2 (a triangle and a 5-cycle);
* ``grid3x2``: the 3 x 2 grid 0-1-2 / 3-4-5 with rungs 0-3, 1-4, 2-5;
* ``path3`` .. ``path5``, ``star4``, ``diamond``, ``tailed_triangle``;
* ``star5`` .. ``star7``: a centre 0 with 4 .. 6 leaves;
* ``three_ears``: the triangle 0-1-2 with vertex 3 on edge 0-1, 4 on 1-2
  and 5 on 0-2 (three pairwise non-adjacent vertices last).
"""

import numpy as np

from .rng import stream, uniform01


def edges_to_adj(k, edges):
    adj = np.zeros((k, k), dtype=np.uint8)
    for a, b in edges:
        adj[a, b] = adj[b, a] = 1
    return adj


def _clique(k):
    return [(a, b) for a in range(k) for b in range(a + 1, k)]


def _cycle(k):
    return [(i, (i + 1) % k) for i in range(k)]


NAMED_PATTERNS = {
    "triangle": (3, _clique(3)),
    "k4": (4, _clique(4)),
    "k5": (5, _clique(5)),
    "k6": (6, _clique(6)),
    "k7": (7, _clique(7)),
    "house": (5, [(0, 1), (1, 2), (2, 3), (3, 0), (2, 4), (3, 4)]),
    "c4": (4, _cycle(4)),
    "c5": (5, _cycle(5)),
    "c6": (6, _cycle(6)),
    "c7": (7, _cycle(7)),
    "k6e": (6, [e for e in _clique(6) if e != (0, 1)]),
    "c6chord": (6, _cycle(6) + [(0, 2)]),
    "grid3x2": (6, [(0, 1), (1, 2), (3, 4), (4, 5), (0, 3), (1, 4), (2, 5)]),
    "path3": (3, [(0, 1), (1, 2)]),
    "path4": (4, [(0, 1), (1, 2), (2, 3)]),
    "path5": (5, [(0, 1), (1, 2), (2, 3), (3, 4)]),
    "star4": (4, [(0, 1), (0, 2), (0, 3)]),
    "diamond": (4, [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3)]),
    "tailed_triangle": (4, [(0, 1), (1, 2), (2, 0), (2, 3)]),
    "star5": (5, [(0, i) for i in range(1, 5)]),
    "star6": (6, [(0, i) for i in range(1, 6)]),
    "star7": (7, [(0, i) for i in range(1, 7)]),
    "three_ears": (6, [(0, 1), (1, 2), (0, 2), (3, 0), (3, 1), (4, 1), (4, 2), (5, 0), (5, 2)]),
}


def named_pattern(name):
    k, edges = NAMED_PATTERNS[name]
    return edges_to_adj(k, edges)


def is_connected(adj):
    """Breadth-first reachability from vertex 0 (input validation only)."""
    k = adj.shape[0]
    seen = {0}
    todo = [0]
    while todo:
        a = todo.pop()
        for b in range(k):
            if adj[a, b] and b not in seen:
                seen.add(b)
                todo.append(b)
    return len(seen) == k


def random_connected_pattern(k, p, seed, index):
    """One random connected pattern on ``k`` vertices.

    Attempt ``t`` of pattern ``index`` draws every pair ``a < b`` in row-major
    order, with counters starting at ``(index * 4096 + t) * 32``; the pair is
    an edge when its uniform draw is below ``p``. Attempts repeat until the
    pattern is connected.
    """
    pairs = [(a, b) for a in range(k) for b in range(a + 1, k)]
    for t in range(4096):
        u = uniform01(stream(seed, (index * 4096 + t) * 32, len(pairs)))
        adj = edges_to_adj(k, [pr for pr, x in zip(pairs, u) if x < p])
        if is_connected(adj):
            return adj
    raise RuntimeError("no connected pattern drawn")


def random_pattern_set(count, k_lo, k_hi, p, seed):
    """``count`` random connected patterns; the size of pattern ``i`` is drawn
    uniformly from ``[k_lo, k_hi]`` with counter ``i`` of stream ``seed + 1``."""
    ku = uniform01(stream(seed + 1, 0, count))
    out = []
    for i in range(count):
        k = k_lo + min(int(ku[i] * (k_hi - k_lo + 1)), k_hi - k_lo)
        out.append(random_connected_pattern(k, p, seed, i))
    return out
