"""The serving loop's host logic on CPU, with a fake of the library: partial
counts over time slices add up exactly, admission respects the memory
budget, and every failure path (a work item over its limit, too many
slices, a planning error, a failing launch) answers the affected requests
with an error while the others complete. No GPU: the fake stands in for
gp_count_batch_ranges and the planner calls."""

import threading
import time

import numpy as np
import pytest

from paper_2009_10955_gb300 import serve


class FakeGraph:
    def __init__(self, nnz):
        self.nnz = nnz

    def device_csr(self):
        return 0, 0, self.nnz


class FakeSched:
    def __init__(self, adj):
        self.k = adj.shape[0]
        self.key = adj.tobytes()

    def set_iep(self, enable=True):
        return 0

    def iep(self, idx=0):
        return 0, 1


class FakeNative:
    """Each slice advances every job by `per_slice` tasks; a task of a
    k-vertex pattern counts k. A pattern with a self loop fails planning; a
    job whose task range reaches `poison_task` is abandoned (next = -1)."""

    def __init__(self, per_slice=7, poison_task=None, fail_launch=False, plan_s=0.0):
        self.plan_s = plan_s
        self.per_slice = per_slice
        self.poison_task = poison_task
        self.fail_launch = fail_launch
        self.max_batch_seen = 0
        self.launches = 0
        self.lock = threading.Lock()

    def gp_pattern_create(self, adj):
        if np.any(np.diag(adj)):
            raise ValueError("bad pattern")
        return adj

    def gp_schedule(self, pattern, graph, top_k=1, stream=None):
        time.sleep(self.plan_s)              # a slow planner
        return FakeSched(pattern)

    def gp_count_scratch_bytes(self, graph, sched, idx):
        return 1000 * sched.k

    def make_opts(self, **kw):
        return kw

    def gp_count_batch_ranges(self, graphs, scheds, idx, begin, end, opts, stream=None, raw=None):
        st, out, nxt = self._ranges(scheds, begin, end)
        if raw is not None:
            raw[0::2] = out
            raw[1::2] = 0
        return st, out, nxt

    def _ranges(self, scheds, begin, end):
        with self.lock:
            self.launches += 1
            self.max_batch_seen = max(self.max_batch_seen, len(scheds))
        if self.fail_launch:
            raise RuntimeError("launch failed")
        out, nxt = [], []
        for s, b, e in zip(scheds, begin, end):
            t = min(e, b + self.per_slice)
            if self.poison_task is not None and b <= self.poison_task < t and s.k == 5:
                out.append(0)
                nxt.append(-1)
                continue
            out.append((t - b) * s.k)
            nxt.append(t)
        return 0, np.array(out, np.uint64), np.array(nxt, np.int64)


def adj_k(k):
    a = np.ones((k, k), np.uint8)
    np.fill_diagonal(a, 0)
    return a


@pytest.fixture
def fake(monkeypatch):
    def make(**kw):
        f = FakeNative(**kw)
        monkeypatch.setattr(serve, "N", f)
        return f
    return make


def wait_all(reqs, timeout=10.0):
    for r in reqs:
        assert r.done.wait(timeout), f"request {r.rid} did not finish"


def test_slices_add_up_exactly(fake):
    f = fake(per_slice=7)
    srv = serve.Server({"a": FakeGraph(100), "b": FakeGraph(31)}, slice_ms=1.0)
    try:
        reqs = [srv.submit("a", adj_k(3)), srv.submit("b", adj_k(4)), srv.submit("a", adj_k(4))]
        wait_all(reqs)
    finally:
        srv.close()
    assert [r.count for r in reqs] == [300, 124, 400]
    assert [r.error for r in reqs] == [None, None, None]
    assert reqs[0].slices == 15 and reqs[1].slices == 5      # ceil(100 / 7), ceil(31 / 7)
    assert f.max_batch_seen >= 2                             # the jobs shared launches


def test_memory_budget_limits_the_batch(fake):
    f = fake(per_slice=5)
    # scratch 1000 k bytes per job; a budget of 3500 admits one 3-vertex job
    # beside nothing larger than itself at a time
    srv = serve.Server({"a": FakeGraph(40)}, slice_ms=1.0, mem_budget=3500)
    try:
        reqs = [srv.submit("a", adj_k(3)) for _ in range(2)] + [srv.submit("a", adj_k(4))]
        wait_all(reqs)
    finally:
        srv.close()
    assert [r.count for r in reqs] == [120, 120, 160]
    assert f.max_batch_seen == 2         # two 3-vertex jobs fit; the 4-vertex job waits
    assert srv.deferrals > 0             # and its admission was put off at least once


def test_abandoned_work_item_times_out_alone(fake):
    fake(per_slice=10, poison_task=25)
    srv = serve.Server({"a": FakeGraph(60)}, slice_ms=1.0, item_ms=1.0)
    try:
        bad = srv.submit("a", adj_k(5))
        good = srv.submit("a", adj_k(3))
        wait_all([bad, good])
    finally:
        srv.close()
    assert isinstance(bad.error, TimeoutError) and bad.count is None
    assert good.error is None and good.count == 180


def test_max_slices_and_deadline(fake):
    fake(per_slice=1)
    srv = serve.Server({"a": FakeGraph(50)}, slice_ms=1.0, max_slices=3)
    try:
        r = srv.submit("a", adj_k(3))
        wait_all([r])
    finally:
        srv.close()
    assert isinstance(r.error, TimeoutError) and r.slices == 3
    fake(per_slice=1)
    srv = serve.Server({"a": FakeGraph(10 ** 9)}, slice_ms=1.0, deadline_s=0.05)
    try:
        r = srv.submit("a", adj_k(3))
        wait_all([r])
    finally:
        srv.close()
    assert isinstance(r.error, TimeoutError) and r.latency >= 0.05


def test_planning_error_answers_only_that_request(fake):
    fake(per_slice=50)
    srv = serve.Server({"a": FakeGraph(20)}, slice_ms=1.0)
    bad_adj = adj_k(3)
    bad_adj[0, 0] = 1
    try:
        bad = srv.submit("a", bad_adj)
        good = srv.submit("a", adj_k(3))
        wait_all([bad, good])
    finally:
        srv.close()
    assert isinstance(bad.error, ValueError)
    assert good.count == 60


def test_failing_launch_answers_the_batch(fake):
    fake(fail_launch=True)
    srv = serve.Server({"a": FakeGraph(20)}, slice_ms=1.0)
    try:
        reqs = [srv.submit("a", adj_k(3)), srv.submit("a", adj_k(4))]
        wait_all(reqs)
        # the server keeps serving after a failed launch
        assert srv.thread.is_alive()
    finally:
        srv.close()
    assert all(isinstance(r.error, RuntimeError) for r in reqs)


class FakeCursor(FakeNative):
    """Models the launch's task order: tasks of the jobs in the order given,
    each costing `cost[k]` units, until the slice budget of `budget` units is
    spent (the task that crosses it still completes)."""

    def __init__(self, budget, cost):
        super().__init__()
        self.budget = budget
        self.cost = cost

    def _ranges(self, scheds, begin, end):
        self.launches += 1
        left = self.budget
        out, nxt = [], []
        for s, b, e in zip(scheds, begin, end):
            t = b
            while t < e and left > 0:
                left -= self.cost[s.k]
                t += 1
            out.append((t - b) * s.k)
            nxt.append(t)
        return 0, np.array(out, np.uint64), np.array(nxt, np.int64)


def test_quota_rule():
    assert serve.next_quota(100, 100, True, 8) == 200           # finished: double
    assert serve.next_quota(100, 40, False, 8) == 20            # cut: half of what it did
    assert serve.next_quota(100, 3, False, 8) == 8              # never below the minimum
    assert serve.next_quota(100, 0, False, 8) == 100            # no progress: unchanged


def test_heavy_jobs_do_not_starve_the_rest(fake, monkeypatch):
    # three 5-vertex jobs whose tasks cost 1000 units each over huge task
    # ranges, submitted first, then light 3-vertex jobs (1 unit per task,
    # 300 tasks); 20,000 units per slice
    f = FakeCursor(budget=20000, cost={5: 1000, 3: 1})
    monkeypatch.setattr(serve, "N", f)
    srv = serve.Server({"big": FakeGraph(10 ** 7), "small": FakeGraph(300)}, slice_ms=1.0,
                       quota0=4096, max_slices=100)
    try:
        heavy = [srv.submit("big", adj_k(5)) for _ in range(3)]
        time.sleep(0.05)
        light = [srv.submit("small", adj_k(3)) for _ in range(4)]
        wait_all(light)
        assert all(r.count == 900 and r.error is None for r in light)
        # the light jobs finished within a few slices of their admission
        assert max(r.slices for r in light) <= 3
    finally:
        srv.close()
    wait_all(heavy)
    assert all(isinstance(r.error, TimeoutError) for r in heavy)    # max_slices
    # the heavy jobs' windows shrank below their first quota
    assert all(r.quota < 4096 for r in heavy)


def test_latency_runs_from_arrival_and_planning_does_not_block_submit(fake):
    """A slow planner: submit() returns at once for every client, and each
    latency is measured from the arrival time (stamped before the lock, or
    given), so it includes the time spent waiting for the planner."""
    fake(per_slice=1000, plan_s=0.2)
    srv = serve.Server({"a": FakeGraph(10)}, slice_ms=1.0)
    try:
        t0 = time.perf_counter()
        reqs, took = [], []
        for k in (3, 4, 5, 6):
            a = time.perf_counter()
            reqs.append(srv.submit("a", adj_k(k)))
            took.append(time.perf_counter() - a)
        given = srv.submit("a", adj_k(7), arrival=t0)
        wait_all(reqs + [given])
    finally:
        srv.close()
    assert max(took) < 0.1                       # never waited for the planner
    assert all(r.arrival >= t0 and r.arrival - t0 < 0.1 for r in reqs)
    # four distinct patterns planned one after another at 0.2 s each: the
    # last one waited behind the others and its latency shows it
    lat = sorted(r.latency for r in reqs)
    assert lat[-1] >= 0.6
    assert given.arrival == t0 and given.latency >= 0.8
    assert [r.count for r in reqs] == [30, 40, 50, 60]


class FakeIepSched(FakeSched):
    """An inclusion-exclusion plan: a 4-vertex pattern divides by 2, a
    5-vertex one by 3 (its fake totals are then not divisible)."""

    def set_iep(self, enable=True):
        return 1

    def iep(self, idx=0):
        return (2, 2) if self.k == 4 else (2, 3) if self.k == 5 else (0, 1)


class FakeIepNative(FakeNative):
    """Slices return undivided 128-bit totals: (tasks x k) x 2 for every
    plan, and 2^64 per task on top for 6-vertex patterns, whose counts then
    need more than 64 bits."""

    def gp_schedule(self, pattern, graph, top_k=1, stream=None):
        return FakeIepSched(pattern)

    def gp_count_batch_ranges(self, graphs, scheds, idx, begin, end, opts, stream=None, raw=None):
        st, out, nxt = self._ranges(scheds, begin, end)
        assert raw is not None
        for j, (s, b, t) in enumerate(zip(scheds, begin, nxt)):
            total = int(out[j]) * 2 + ((int(t) - b) << 64 if s.k == 6 else 0)
            raw[2 * j], raw[2 * j + 1] = total & ((1 << 64) - 1), total >> 64
            out[j] = 0                                  # partial IEP totals are not counts
        return st, out, nxt


def test_inclusion_exclusion_totals_divided_once(monkeypatch):
    f = FakeIepNative(per_slice=7)
    monkeypatch.setattr(serve, "N", f)
    srv = serve.Server({"a": FakeGraph(100)}, slice_ms=1.0, iep=True)
    try:
        reqs = [srv.submit("a", adj_k(k)) for k in (3, 4, 5, 6)]
        wait_all(reqs)
    finally:
        srv.close()
    # 3 vertices: divisor 1, raw = 2 x count of the fake; 4: divisor 2
    assert reqs[0].count == 600 and reqs[0].error is None
    assert reqs[1].count == 400 and reqs[1].error is None
    # 5 vertices: 100 x 5 x 2 = 1000 is not a multiple of 3; 6: beyond 64 bits
    assert reqs[2].count is None and isinstance(reqs[2].error, ArithmeticError)
    assert reqs[3].count is None and isinstance(reqs[3].error, ArithmeticError)
    assert reqs[1].slices == 15
