"""Continuous-batching server for pattern-count queries on device-resident
graphs.

Requests (graph name, pattern) arrive at any time. The server keeps the
graphs and the plans on the device and runs in time slices: each slice is
ONE persistent launch (``gp_count_batch_ranges``) over every admitted job,
cut off after ``slice_cycles`` device cycles. Between slices, finished jobs
leave, their results are published, and requests that arrived meanwhile are
admitted as long as the slice's intermediate-set scratch stays within the
memory budget. A job's partial counts over disjoint task ranges add up to
its exact count, so a job may span any number of slices.

The launch hands out the jobs' edge tasks in job order, so a job with
expensive tasks at the front of the order could take a whole slice from the
jobs behind it. Each job therefore gets a task window per slice (its quota):
the quota doubles while the job finishes its window inside the slice and
halves below what the job managed when the slice ended first (leaving the
rest of the next slice to the others); and the job order rotates from slice
to slice, so that every job is at the front in turn.

Plans use inclusion-exclusion for their innermost loops where it applies
(Section IV-D); a slice then returns each job's undivided 128-bit partial
total, the partial totals add up over the slices, and the request's count is
their sum divided by the plan's divisor.

Planning (and sizing a request's scratch) runs in the server thread without
holding the lock that submit() takes, so clients are never blocked behind the
planner, and a request's latency runs from the arrival time stamped before
submit() takes that lock (or given by the caller).

The scheduling here is host-side bookkeeping; all counting runs in the
library's kernels.
"""

import collections
import threading
import time

import numpy as np

from . import _native as N


def next_quota(quota, done, finished_window, quota_min):
    """Task window of a job for its next slice: double it after a window
    the job finished inside the slice, half of what it managed when the
    slice ended first, unchanged when it made no progress (it was behind
    other jobs; the rotation brings it forward)."""
    if finished_window:
        return min(2 * quota, 1 << 40)
    if done > 0:
        return max(quota_min, done // 2)
    return quota


class Request:
    __slots__ = ("rid", "graph", "adj", "arrival", "done", "count", "error", "finish", "sched",
                 "next_task", "end_task", "acc", "slices", "scratch", "quota", "div")

    def __init__(self, rid, graph, adj, arrival):
        self.rid = rid
        self.graph = graph
        self.adj = np.ascontiguousarray(adj, dtype=np.uint8)
        self.arrival = arrival
        self.done = threading.Event()
        self.count = None
        self.error = None
        self.finish = None
        self.sched = None
        self.next_task = 0
        self.end_task = 0
        self.acc = 0
        self.slices = 0
        self.scratch = 0
        self.quota = 0
        self.div = 1

    @property
    def latency(self):
        return None if self.finish is None else self.finish - self.arrival


class Server:
    """Continuous batching over device-resident graphs (see module doc)."""

    def __init__(self, graphs, slice_ms=20.0, max_batch=256, mem_budget=None, stream=None,
                 clock_ghz=1.9, max_slices=None, item_ms=None, deadline_s=None, quota0=4096,
                 quota_min=64, iep=True):
        self.graphs = dict(graphs)
        self.slice_cycles = int(slice_ms * 1e-3 * clock_ghz * 1e9)
        # with item_ms, a single work item (edge task) that needs longer than
        # that abandons its request with a timeout, so that a slice cannot
        # outlive its budget by more than item_ms
        self.item_cycles = int(item_ms * 1e-3 * clock_ghz * 1e9) if item_ms else 0
        self.max_batch = max_batch
        self.mem_budget = mem_budget
        self.stream = stream
        self.max_slices = max_slices
        self.deadline_s = deadline_s      # wall-clock limit per request (from arrival)
        self.quota0 = quota0              # first task window of a job (tasks per slice)
        self.quota_min = quota_min
        self.iep = iep                    # inclusion-exclusion where a plan qualifies
        self._plans = {}
        self._pending = collections.deque()
        self._active = []
        self._cv = threading.Condition()
        self._stop = False
        self._rid = 0
        self._nnz = {k: g.device_csr()[2] for k, g in self.graphs.items()}
        self.slices = 0
        self.deferrals = 0                # admissions put off by the memory budget
        self.thread = threading.Thread(target=self._loop, daemon=True)
        self.thread.start()

    # ------------------------------------------------------------ client side
    def submit(self, graph, adj, arrival=None):
        """Queue a request. Its latency runs from `arrival` (perf_counter
        seconds), stamped here before any lock is taken when not given."""
        t = time.perf_counter() if arrival is None else arrival
        with self._cv:
            self._rid += 1
            r = Request(self._rid, graph, adj, t)
            self._pending.append(r)
            self._cv.notify()
        return r

    def close(self):
        with self._cv:
            self._stop = True
            self._cv.notify()
        self.thread.join()

    # ------------------------------------------------------------ server side
    def _plan(self, graph, adj):
        key = (graph, adj.tobytes(), adj.shape[0])
        s = self._plans.get(key)
        if s is None:
            g = self.graphs[graph]
            s = N.gp_schedule(N.gp_pattern_create(adj), g, top_k=1, stream=self.stream)
            if self.iep:
                s.set_iep(True)
            self._plans[key] = s
        return s

    def _admit(self):
        """Move pending requests into the active set while the batch's
        scratch (the maximum over its jobs) fits the memory budget. The
        candidates are taken under the lock, planned and sized without it,
        and admitted (in arrival order) under it again."""
        with self._cv:
            room = self.max_batch - len(self._active)
            cand = [self._pending.popleft() for _ in range(min(room, len(self._pending)))]
        planned = []
        for r in cand:
            try:
                r.sched = self._plan(r.graph, r.adj)
                r.scratch = N.gp_count_scratch_bytes(self.graphs[r.graph], r.sched, 0)
                r.div = r.sched.iep(0)[1]
            except Exception as e:  # bad pattern or graph: answer with the error
                r.error = e
                r.finish = time.perf_counter()
                r.done.set()
                continue
            planned.append(r)
        with self._cv:
            back = []
            for r in planned:
                need = max([a.scratch for a in self._active] + [r.scratch])
                if back or (self.mem_budget is not None and self._active and need > self.mem_budget):
                    back.append(r)              # waits, and so does every later request
                    continue
                r.next_task, r.end_task = 0, self._nnz[r.graph]
                r.quota = self.quota0
                self._active.append(r)
            self._pending.extendleft(reversed(back))
            self.deferrals += len(back)

    def _loop(self):
        while True:
            with self._cv:
                while not self._stop and not self._pending and not self._active:
                    self._cv.wait()
                if self._stop and not self._pending and not self._active:
                    return
            self._admit()
            with self._cv:
                batch = list(self._active)
            if not batch:
                continue
            rot = self.slices % len(batch)              # every job at the front in turn
            batch = batch[rot:] + batch[:rot]
            window = [min(r.end_task, r.next_task + r.quota) for r in batch]
            opts = N.make_opts(budget_cycles=self.slice_cycles, task_cycles=self.item_cycles)
            raw = np.zeros(2 * len(batch), dtype=np.uint64)
            try:
                st, out, nxt = N.gp_count_batch_ranges(
                    [self.graphs[r.graph] for r in batch], [r.sched for r in batch],
                    [0] * len(batch), [r.next_task for r in batch], window,
                    opts, stream=self.stream, raw=raw)
            except Exception as e:
                now = time.perf_counter()
                with self._cv:
                    for r in batch:
                        r.error, r.finish = e, now
                        r.done.set()
                    self._active = []
                continue
            self.slices += 1
            now = time.perf_counter()
            with self._cv:
                still = []
                for j, (r, t, w) in enumerate(zip(batch, nxt, window)):
                    r.slices += 1
                    if int(t) < 0:                       # a work item outlived item_cycles
                        r.error = TimeoutError(f"request {r.rid}: a work item exceeded the item limit")
                        r.finish = now
                        r.done.set()
                        continue
                    r.acc += int(raw[2 * j]) | (int(raw[2 * j + 1]) << 64)
                    r.quota = next_quota(r.quota, int(t) - r.next_task, int(t) >= w, self.quota_min)
                    r.next_task = int(t)
                    if r.next_task >= r.end_task:
                        if r.acc % r.div or (r.acc // r.div) >> 64:
                            r.error = ArithmeticError(f"request {r.rid}: total {r.acc} is not a 64-bit "
                                                      f"multiple of its divisor {r.div}")
                        else:
                            r.count = r.acc // r.div
                        r.finish = now
                        r.done.set()
                    elif self.max_slices is not None and r.slices >= self.max_slices:
                        r.error = TimeoutError(f"request {r.rid} exceeded {self.max_slices} slices")
                        r.finish = now
                        r.done.set()
                    elif self.deadline_s is not None and now - r.arrival > self.deadline_s:
                        r.error = TimeoutError(f"request {r.rid} exceeded its {self.deadline_s} s deadline")
                        r.finish = now
                        r.done.set()
                    else:
                        still.append(r)
                order = {id(r): i for i, r in enumerate(self._active)}
                self._active = sorted(still, key=lambda r: order[id(r)])


def poisson_arrivals(rate, count, seed):
    """Arrival offsets (seconds) of a Poisson process, from the project PRNG."""
    from synth.rng import stream, uniform01
    u = uniform01(stream(seed, 0, count))
    return np.cumsum(-np.log1p(-u) / rate)
