"""Directed patterns on directed graphs through the C ABI against the
oracle's directed enumeration (a reading: every pattern arc must map to a
graph arc; counts divide by the arc-preserving automorphisms)."""

import numpy as np
import pytest

import oracle
from oracle import planner_ref as pr
from synth.rng import stream

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def N():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2009_10955_gb300 import native
    return native()


def pat(k, arcs):
    a = np.zeros((k, k), np.uint8)
    for x, y in arcs:
        a[x, y] = 1
    return a


PATTERNS = {
    "cycle3": pat(3, [(0, 1), (1, 2), (2, 0)]),
    "path3": pat(3, [(0, 1), (1, 2)]),
    "feed_forward": pat(3, [(0, 1), (0, 2), (1, 2)]),
    "mutual_triangle": pat(3, [(a, b) for a in range(3) for b in range(3) if a != b]),
    "cycle4": pat(4, [(0, 1), (1, 2), (2, 3), (3, 0)]),
    "bifan": pat(4, [(0, 2), (0, 3), (1, 2), (1, 3)]),
    "mixed4": pat(4, [(0, 1), (1, 0), (1, 2), (3, 2), (0, 3)]),
    "out_star4": pat(4, [(0, 1), (0, 2), (0, 3)]),
    "cycle5": pat(5, [(i, (i + 1) % 5) for i in range(5)]),
}


def arcs(n, m, seed, skew=False):
    u = stream(seed, 0, 2 * m)
    if skew:        # many arcs at low ids: hub-like vertices
        x = (u >> np.uint64(11)).astype(np.float64) / float(1 << 53)
        ids = np.minimum((x ** 3 * n).astype(np.int64), n - 1)
    else:
        ids = (u % np.uint64(n)).astype(np.int64)
    p = ids.reshape(m, 2)
    return p[:, 0].astype(np.int32), p[:, 1].astype(np.int32)


@pytest.mark.parametrize("n,m,seed,skew", [(60, 700, 1, False), (300, 2500, 2, True)])
def test_lists_bit_exact(N, n, m, seed, skew):
    s, d = arcs(n, m, seed, skew)
    g = N.gp_dgraph_create(s, d, n)
    ref = oracle.build_dcsr(n, s, d)
    op, oc, ip, ic = g.lists()
    assert np.array_equal(op, ref.out_ptr) and np.array_equal(oc, ref.out_col)
    assert np.array_equal(ip, ref.in_ptr) and np.array_equal(ic, ref.in_col)
    assert g.stats() == {"n": n, "narcs": ref.narcs}


@pytest.mark.parametrize("name", sorted(PATTERNS))
@pytest.mark.parametrize("n,m,seed,skew", [(60, 700, 1, False), (300, 2500, 2, True)])
def test_count_equals_oracle(N, name, n, m, seed, skew):
    s, d = arcs(n, m, seed, skew)
    g = N.gp_dgraph_create(s, d, n)
    ref = oracle.build_dcsr(n, s, d)
    p = PATTERNS[name]
    truth = oracle.count_directed(p, ref)
    dp = N.gp_dpattern_create(p)
    assert N.gp_dcount(g, dp) == truth
    # explicit configurations: efficient schedules with Algorithm 1's sets,
    # and without restrictions (divided by |Aut|)
    al = p.tolist()
    scheds, _ = pr.efficient_schedules(al)
    sets = pr.restriction_sets(al)
    for sc in scheds[:3]:
        assert N.gp_dcount(g, dp, order=sc, restrictions=[]) == truth
        for rs in sets[:2]:
            assert N.gp_dcount(g, dp, order=sc, restrictions=list(rs)) == truth


def test_edge_cases(N):
    dp = N.gp_dpattern_create(PATTERNS["cycle3"])
    empty = N.gp_dgraph_create(np.zeros(0, np.int32), np.zeros(0, np.int32), 0)
    assert N.gp_dcount(empty, dp) == 0
    loops = N.gp_dgraph_create(np.arange(5, dtype=np.int32), np.arange(5, dtype=np.int32), 5)
    assert loops.stats()["narcs"] == 0 and N.gp_dcount(loops, dp) == 0
    ring = N.gp_dgraph_create(np.array([0, 1, 2], np.int32), np.array([1, 2, 0], np.int32), 3)
    assert N.gp_dcount(ring, dp) == 1
    rev = N.gp_dgraph_create(np.array([0, 1, 0], np.int32), np.array([1, 2, 2], np.int32), 3)
    assert N.gp_dcount(rev, dp) == 0
    with pytest.raises(N.GraphPiError) as e:
        N.gp_dgraph_create(np.array([0], np.int32), np.array([5], np.int32), 3)
    assert e.value.status == N.GP_ERR_ARG
    with pytest.raises(N.GraphPiError) as e:                    # not a valid set for the 3-cycle
        N.gp_dcount(ring, dp, order=(0, 1, 2), restrictions=[(0, 1)])
    assert e.value.status == N.GP_ERR_PATTERN
