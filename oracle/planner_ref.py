"""Plain restatement of GraphPi's configuration generation and performance
model (Sections IV-A to IV-C), for checking the library's C++ planner.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Notation follows the paper. A pattern is a k x k symmetric 0/1 matrix over
vertices 0..k-1. A permutation ``perm`` is a tuple with ``perm[v]`` the image
of ``v``. A restriction ``(a, b)`` means id(a) > id(b). A schedule is the
tuple of pattern vertices in search order; loops are numbered 1..n as in the
paper's performance model.

Readings of the paper used here (where the text is silent or garbled):

* Algorithm 1 finds a 2-cycle as a vertex that is the image of its own
  image; a fixed point also meets that test, so the vertex must also differ
  from its image, and the pair added is ``(vertex, perm[vertex])``.
* The elimination explores restriction sets, not permutation groups: the
  automorphisms a branch still has to eliminate are exactly those that
  survive its set under ``no_conflict``, which is monotone (a permutation
  that closes a cycle under a set still closes it under every superset), so
  every set needs to be examined once.
* Phase 2 of the schedule filter can leave no schedule at all (for example
  the 4-cycle and 6-cycle); the largest k' <= k that keeps at least one
  phase-1 schedule is used instead, and k' = 1 means phase 1 alone.
* ``|E|`` counts undirected edges; ``tri_cnt`` counts each triangle once per
  ordered vertex triple (six times per triangle), so that
  ``|V| p1 p2 = tri_cnt / (2|E|)`` is the mean common-neighbour count of a
  directed edge, matching the stated meaning of ``p2``.
* A restriction acts in the loop of its later-scheduled endpoint. ``f_i`` is
  the fraction of the relative orders still alive at loop i that the
  restrictions of loop i remove (0 when loop i has none).
* ``c_i`` sums, over the distinct partial intersections computed in loop i,
  the estimated sizes of its two operands: the partial set built so far
  and ``N(v_i)``. A vertex whose candidate set has operands at loops
  ``j1 < j2 < ... < jm`` gets ``N(v_j1) ∩ N(v_j2)`` in loop j2, that result
  intersected with ``N(v_j3)`` in loop j3, and so on; equal partial sets
  (same operand loops) are computed once.
"""

from itertools import combinations, permutations
from math import factorial


def _edges(adj):
    k = len(adj)
    return [(a, b) for a in range(k) for b in range(k) if adj[a][b]]


def automorphisms(adj, labels=None):
    """All permutations preserving the edge set (Section IV-A), and the
    vertex labels when the pattern is labelled."""
    k = len(adj)
    E = _edges(adj)
    return [p for p in permutations(range(k)) if all(adj[p[a]][p[b]] for a, b in E)
            and (labels is None or all(labels[p[a]] == labels[a] for a in range(k)))]


def _acyclic(k, arcs):
    """Kahn's algorithm on a directed graph over 0..k-1."""
    indeg = [0] * k
    out = [[] for _ in range(k)]
    for a, b in arcs:
        out[a].append(b)
        indeg[b] += 1
    ready = [v for v in range(k) if indeg[v] == 0]
    seen = 0
    while ready:
        v = ready.pop()
        seen += 1
        for w in out[v]:
            indeg[w] -= 1
            if indeg[w] == 0:
                ready.append(w)
    return seen == k


def no_conflict(perm, res_set):
    """True when ``perm`` is NOT eliminated by ``res_set``: the digraph with
    arcs first->second and perm[first]->perm[second] for every restriction is
    acyclic (Algorithm 1, no_conflict)."""
    arcs = []
    for a, b in res_set:
        arcs.append((a, b))
        arcs.append((perm[a], perm[b]))
    return _acyclic(len(perm), arcs)


def linear_extensions(k, res_set):
    """Orderings of k distinct labels obeying every restriction: the
    restricted embedding count of the pattern in the k-vertex complete graph."""
    return sum(1 for sigma in permutations(range(k))
               if all(sigma[a] > sigma[b] for a, b in res_set))


def validate(k, aut_count, res_set):
    """ans_with == ans_without / |Aut| on the k-vertex complete graph, where
    ans_without = k! (every injective map is an embedding there)."""
    return linear_extensions(k, res_set) * aut_count == factorial(k)


def restriction_sets(adj, labels=None):
    """The restriction sets of Section IV-A's 2-cycle elimination
    (Algorithm 1), as a sorted list of sorted tuples of pairs.

    Restated as a breadth-first search over restriction sets, level by level
    in the number of restrictions. A set that some automorphism other than
    the identity survives (``no_conflict``) is extended, once for every
    2-cycle (v, w) of every surviving automorphism, by the restriction
    (v, w); a set that only the identity survives is final, and it is kept
    when its linear extensions times |Aut| equal k! (``validate``). Each set
    is visited once however many routes lead to it."""
    k = len(adj)
    auts = automorphisms(adj, labels)
    n_aut = len(auts)
    level = {frozenset()}
    seen = set(level)
    found = set()
    while level:
        following = set()
        for res_set in level:
            alive = [p for p in auts if no_conflict(p, res_set)]
            if len(alive) <= 1:
                if validate(k, n_aut, res_set):
                    found.add(res_set)
                continue
            for perm in alive:
                for v in range(k):
                    w = perm[v]
                    if w != v and perm[w] == v:                     # a 2-cycle (v, w)
                        child = res_set | {(v, w)}
                        if child not in seen:
                            seen.add(child)
                            following.add(child)
        level = following
    return sorted(tuple(sorted(s)) for s in found)


def max_independent_set_size(adj):
    k = len(adj)
    for size in range(k, 0, -1):
        for sub in combinations(range(k), size):
            if all(not adj[a][b] for a, b in combinations(sub, 2)):
                return size
    return 0


def phase1_ok(adj, sched):
    """Every vertex after the first is adjacent to an earlier one, i.e. every
    prefix induces a connected subgraph (Section IV-B, phase 1)."""
    return all(any(adj[sched[i]][sched[j]] for j in range(i)) for i in range(1, len(sched)))


def phase2_ok(adj, sched, kk):
    """The last kk searched vertices are pairwise non-adjacent (phase 2)."""
    tail = sched[len(sched) - kk:]
    return all(not adj[a][b] for a, b in combinations(tail, 2))


def underlying(adj):
    """The undirected pattern under a directed one (an edge wherever an arc
    runs either way); an undirected pattern is its own."""
    k = len(adj)
    return [[1 if (adj[a][b] or adj[b][a]) else 0 for b in range(k)] for a in range(k)]


def efficient_schedules(adj):
    """(schedules, k') : the 2-phase filter with phase 2 relaxed to the
    largest k' that keeps a schedule. For a directed pattern both phases
    look at its underlying undirected pattern (a vertex joined to an earlier
    one by an arc of either direction has its candidates in that vertex's
    out- or in-list)."""
    adj = underlying(adj)
    k = len(adj)
    p1 = [s for s in permutations(range(k)) if phase1_ok(adj, s)]
    for kk in range(max_independent_set_size(adj), 0, -1):
        out = [s for s in p1 if phase2_ok(adj, s, kk)]
        if out:
            return out, kk
    return p1, 1


def graph_params(n_vertices, n_edges, tri_cnt):
    """p1 and p2 of Section IV-C (|E| undirected, tri_cnt ordered)."""
    V, E = float(n_vertices), float(n_edges)
    p1 = 2.0 * E / (V * V)
    p2 = tri_cnt * V / ((2.0 * E) ** 2)
    return p1, p2


def f_values(k, sched, res_set):
    """f_1..f_n by filtering all k! relative orders loop by loop."""
    pos = {v: i for i, v in enumerate(sched)}
    alive = list(permutations(range(k)))
    f = []
    for i in range(k):
        here = [(a, b) for a, b in res_set if max(pos[a], pos[b]) == i]
        before = len(alive)
        for a, b in here:
            alive = [s for s in alive if s[a] > s[b]]
        f.append(0.0 if not here or before == 0 else (before - len(alive)) / before)
    return f


def cost(adj, sched, res_set, n_vertices, n_edges, tri_cnt):
    """cost_1 of the nested performance model for one configuration."""
    k = len(adj)
    V = float(n_vertices)
    p1, p2 = graph_params(n_vertices, n_edges, tri_cnt)

    def card(m):                      # m-way intersection of neighbourhoods
        return V if m == 0 else V * p1 * p2 ** (m - 1)

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
                c[i] += card(len(prefix) - 1) + card(1)
    f = f_values(k, sched, res_set)
    total = l[k - 1] * (1.0 - f[k - 1])
    for i in range(k - 2, -1, -1):
        total = l[i] * (1.0 - f[i]) * (c[i] + total)
    return total


def all_configurations(adj, n_vertices, n_edges, tri_cnt):
    """Every (cost, schedule, restriction set) over the efficient schedules and
    Algorithm 1's sets, sorted by cost, then schedule, then set."""
    scheds, _ = efficient_schedules(adj)
    sets = restriction_sets(adj)
    rows = [(cost(adj, s, r, n_vertices, n_edges, tri_cnt), s, r) for s in scheds for r in sets]
    rows.sort()
    return rows


def components(k, pairs):
    """Connected components of the undirected graph on vertices 1..k whose
    edges are `pairs` (Algorithm 2's partition step), each a sorted list,
    ordered by smallest member."""
    parent = list(range(k + 1))

    def find(a):
        while parent[a] != a:
            a = parent[a]
        return a
    for i, j in pairs:
        ri, rj = find(i), find(j)
        if ri != rj:
            parent[max(ri, rj)] = min(ri, rj)
    comps = {}
    for v in range(1, k + 1):
        comps.setdefault(find(v), []).append(v)
    return sorted(comps.values())


def intersection_card(k, pairs, sets):
    """Algorithm 2: |A_{i1,j1} ∩ ... ∩ A_{im,jm}|, the number of tuples with
    e_l in S_l for every l and e_i = e_j for every listed pair. Each connected
    component of the pairs must take one common value from the intersection of
    its sets; the components choose independently. `sets[l - 1]` is S_l."""
    card = 1
    for comp in components(k, pairs):
        common = set(sets[comp[0] - 1])
        for v in comp[1:]:
            common &= set(sets[v - 1])
        card *= len(common)
    return card


def iep_count(sets):
    """|S_IEP| of Section IV-D: tuples (e_1, ..., e_k), e_l in S_l, with
    pairwise distinct entries, by inclusion-exclusion over every subset of
    the pairs (i, j), i < j, each term from Algorithm 2."""
    k = len(sets)
    all_pairs = [(i, j) for i in range(1, k + 1) for j in range(i + 1, k + 1)]
    total = 0
    for m in range(len(all_pairs) + 1):
        for sub in combinations(all_pairs, m):
            total += (-1) ** m * intersection_card(k, sub, sets)
    return total

