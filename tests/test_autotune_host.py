"""The plan choice's host logic on CPU (autotune.choose_plan) with a fake of
the library: every candidate (the model's top plans, their mirror images,
each with and without inclusion-exclusion where it applies) is counted on
the same task sample; the one with the smallest busy-cycle projection wins,
a candidate whose sample launch stopped early is dropped, and the choice is
cached per graph and pattern."""

import json

import numpy as np
import pytest

from paper_2009_10955_gb300 import autotune


class FakeGraph:
    def __init__(self, nnz):
        self.nnz = nnz

    def stats(self, with_triangles=False):
        return {"n": 1000, "m": self.nnz // 2, "max_deg": 77}

    def device_csr(self):
        return 0, 0, self.nnz


class FakeSched:
    def __init__(self, order, res):
        self.order, self.res, self.iep_on = tuple(order), tuple(map(tuple, res)), False

    def set_iep(self, enable=True):
        self.iep_on = bool(enable) and self.res != ((1, 0),)   # one plan has no IEP form
        return int(self.iep_on)

    def iep(self, idx=0):
        return (2, 1) if self.iep_on else (0, 1)

    def get(self, i):
        return self.order, self.res, 0.0


class FakeTop:
    def __init__(self, plans):
        self.plans = plans

    def __len__(self):
        return len(self.plans)

    def get(self, i):
        order, res = self.plans[i]
        return order, res, float(i)


class FakeNative:
    """Busy cycles per sampled task depend on the candidate: `cost` maps
    (order, restrictions, iep) to cycles per task; a candidate mapped to None
    stops at its budget (GP_PARTIAL)."""
    GP_OK, GP_PARTIAL = 0, 1

    def __init__(self, top, cost):
        self.top, self.cost, self.launches = top, cost, 0

    def gp_pattern_create(self, adj):
        return adj

    def gp_schedule(self, pattern, graph, top_k=3, stream=None):
        return FakeTop(self.top[:top_k])

    def gp_schedule_explicit(self, pattern, order, res):
        return FakeSched(order, res)

    def make_opts(self, **kw):
        return kw

    def gp_count_batch_ranges(self, graphs, scheds, idx, begin, end, opts, stream=None, raw=None):
        self.launches += 1
        s = scheds[0]
        per_task = self.cost[(s.order, s.res, s.iep_on)]
        tasks = sum(int(e) - int(b) for b, e in zip(begin, end))
        busy = opts["busy_cycles"]
        if per_task is None:
            busy[0], busy[1] = 10 ** 9, 64
            return self.GP_PARTIAL, np.zeros(len(scheds), np.uint64), np.array(begin, np.int64)
        busy[0], busy[1] = per_task * tasks, 64
        return self.GP_OK, np.zeros(len(scheds), np.uint64), np.array(end, np.int64)


TOP = [((0, 1, 2), ((0, 1),)), ((0, 2, 1), ((0, 2),))]


def cost_table(best):
    """Cycles per task of every candidate; `best` gets the fewest."""
    cands = []
    for order, res in TOP:
        for r in (res, tuple((b, a) for a, b in res)):
            for iep in (False, True):
                if iep and r == ((1, 0),):
                    continue
                cands.append((order, r, iep))
    table = {c: 1000 + 10 * i for i, c in enumerate(cands)}
    table[best] = 10
    return table


@pytest.fixture
def fake(monkeypatch):
    def make(best, stopped=()):
        cost = cost_table(best)
        for c in stopped:
            cost[c] = None
        f = FakeNative(TOP, cost)
        monkeypatch.setattr(autotune, "N", f)
        return f
    return make


def test_fastest_candidate_wins_and_is_cached(fake, tmp_path):
    best = ((0, 2, 1), ((2, 0),), True)                 # a mirror image, with IEP
    f = fake(best)
    cache = str(tmp_path / "c.json")
    adj = np.ones((3, 3), np.uint8) - np.eye(3, dtype=np.uint8)
    sched, table = autotune.choose_plan(FakeGraph(10000), adj, top_k=2, cache_path=cache, device="fake")
    assert (sched.order, sched.res, sched.iep_on) == best
    # every candidate was counted once: 2 plans x 2 orientations x (plain, IEP) minus the one without IEP
    assert f.launches == len(table) == 7
    times = [t for *_, t in table]
    chosen = [t for o, r, kk, t in table if (tuple(o), tuple(map(tuple, r)), kk > 0) == best]
    assert chosen == [min(times)]
    # the projection: busy cycles x (all tasks / sampled tasks) / (warps x clock)
    done = sum(b - a for a, b in autotune.sample_ranges(10000, 256, 64))
    assert min(times) == pytest.approx(10 * done * (10000 / done) / (64 * 2.07e9))
    # cached: no launch the second time, same choice and table
    f.launches = 0
    sched2, table2 = autotune.choose_plan(FakeGraph(10000), adj, top_k=2, cache_path=cache, device="fake")
    assert f.launches == 0 and (sched2.order, sched2.res, sched2.iep_on) == best
    assert table2 == json.loads(json.dumps(table))


def test_stopped_candidates_are_dropped(fake):
    best = ((0, 1, 2), ((0, 1),), False)
    f = fake(best, stopped=[best])                      # the would-be winner stops at its budget
    adj = np.ones((3, 3), np.uint8) - np.eye(3, dtype=np.uint8)
    sched, table = autotune.choose_plan(FakeGraph(10000), adj, top_k=2, device="fake")
    assert (sched.order, sched.res, sched.iep_on) != best
    assert sum(t is None for *_, t in table) == 1
    finite = [t for *_, t in table if t is not None]
    chosen = [t for o, r, kk, t in table
              if (tuple(o), tuple(map(tuple, r)), kk > 0) == (sched.order, sched.res, sched.iep_on)]
    assert chosen and chosen[0] == min(finite)


def test_nothing_finishes_falls_back_to_the_model(fake):
    f = fake(((0, 1, 2), ((0, 1),), False))
    for c in list(f.cost):
        f.cost[c] = None
    adj = np.ones((3, 3), np.uint8) - np.eye(3, dtype=np.uint8)
    sched, table = autotune.choose_plan(FakeGraph(10000), adj, top_k=2, device="fake")
    assert (sched.order, sched.res) == TOP[0] and not sched.iep_on
    assert all(t is None for *_, t in table)
