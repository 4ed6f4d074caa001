"""Reading R14 on the CPU: the count kernel evaluates Section IV-D's
inclusion-exclusion sum grouped by set partition,
    sum over partitions pi of {1..kk} of
        prod over blocks B of (-1)^(|B|-1) (|B|-1)! |intersection of S_i, i in B|,
walking the partitions as restricted growth strings (g_0 = 0, g_i <= 1 +
max of the earlier entries). This restates that grouping in Python, apart
from the kernel, and checks it against the paper's form (every subset of
the pairs with sign (-1)^m, Algorithm 2 for each term, in the oracle's
planner restatement) and against brute force over distinct tuples. The
per-element mask tally the kernel uses for the intersection sizes is
checked the same way."""

import itertools
from math import factorial

import numpy as np
import pytest

from oracle import planner_ref as pr


def growth_strings(kk):
    """Every restricted growth string of length kk, in the order the
    kernel's successor step produces them (the last entry that can grow is
    incremented and the entries after it reset)."""
    g = [0] * kk
    while True:
        yield list(g)
        i = kk - 1
        while i >= 1:
            if g[i] <= max(g[:i]):
                g[i] += 1
                for j in range(i + 1, kk):
                    g[j] = 0
                break
            i -= 1
        if i < 1:
            return


def partition_sum(card, kk):
    """card(mask) = |intersection of the sets whose bits are in mask|."""
    total = 0
    for g in growth_strings(kk):
        term = 1
        for b in range(max(g) + 1):
            mask = sum(1 << i for i in range(kk) if g[i] == b)
            m = bin(mask).count("1")
            mu = (-1) ** (m - 1) * factorial(m - 1)
            term *= mu * card(mask)
        total += term
    return total


def mask_tally_cards(sets):
    """Intersection sizes as the kernel derives them: each element of a set
    other than the largest gets the mask of the sets holding it, counted at
    the first iterated set that holds it; superset sums over those tallies
    give every |intersection over T| for |T| >= 2; single sets use |S_i|."""
    kk = len(sets)
    big = max(range(kk), key=lambda i: len(sets[i]))
    cnt = [0] * (1 << kk)
    for i in range(kk):
        if i == big:
            continue
        for x in sorted(sets[i]):
            mask = sum(1 << j for j in range(kk) if x in sets[j])
            if any(j < i and j != big and x in sets[j] for j in range(kk)):
                continue
            if bin(mask).count("1") >= 2:
                cnt[mask] += 1
    card = {}
    for t in range(1, 1 << kk):
        if bin(t).count("1") == 1:
            card[t] = len(sets[t.bit_length() - 1])
        else:
            card[t] = sum(cnt[m] for m in range(1 << kk) if m & t == t)
    return card


def brute(sets):
    return sum(1 for t in itertools.product(*[sorted(s) for s in sets]) if len(set(t)) == len(t))


def test_growth_strings_are_the_set_partitions():
    bell = {1: 1, 2: 2, 3: 5, 4: 15, 5: 52}
    for kk, b in bell.items():
        gs = list(growth_strings(kk))
        assert len(gs) == b
        blocks = {frozenset(frozenset(i for i in range(kk) if g[i] == v) for v in set(g)) for g in gs}
        assert len(blocks) == b


@pytest.mark.parametrize("kk", [2, 3, 4, 5])
def test_partition_grouping_equals_pair_subsets_and_brute_force(kk):
    rng = np.random.default_rng(kk)
    for trial in range(25 if kk < 5 else 8):
        u = int(rng.integers(3, 12))
        sets = [set(rng.choice(u, size=int(rng.integers(0, u + 1)), replace=False).tolist()) for _ in range(kk)]
        exact = {t: len(set.intersection(*[sets[i] for i in range(kk) if t >> i & 1])) for t in range(1, 1 << kk)}
        grouped = partition_sum(lambda t: exact[t], kk)
        assert grouped == brute(sets)
        if kk <= 4:                           # 2^10 pair subsets at kk = 5: brute force suffices
            assert grouped == pr.iep_count(sets)
        tally = mask_tally_cards(sets)
        assert tally == exact
