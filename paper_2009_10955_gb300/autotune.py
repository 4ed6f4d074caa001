"""Autotuner for the counting kernel's launch knobs.

Knobs (all fields of ``gp_count_opts``):

* ``blocks_per_sm`` -- resident 8-warp blocks per SM, which selects the
  register budget of the kernel build (2: ~100, 3: 80, 4: 64 registers);
* ``lane_work`` -- probe/merge steps above which a lane hands its last-level
  count to the whole warp (the split between the per-lane and the
  warp-cooperative intersection);
* ``GP_COUNT_NO_CORE`` -- whether intersections may use the core bit matrix
  (bit probes) or always binary-search (the intersection variant);
* ``chunk`` -- edge tasks per work-queue grab outside the high-degree prefix;
* ``split`` -- parts each high-degree-prefix task is cut into (the
  second-level split depth of the work decomposition).

A configuration is timed (CUDA events around the kernel, inside the library)
on a stratified sample of the edge tasks: ``windows`` evenly spaced windows
of ``width`` consecutive tasks, all counted in ONE launch of
``gp_count_batch_ranges``. The best configuration is cached per (device,
graph statistics, plan) in a JSON file.

``choose_plan`` applies the same sampling one level up, to the plan itself:
the performance model (Section IV-C) sees only |V|, |E| and the triangle
count, so it scores a restriction set and its mirror image (every
restriction reversed) identically, although on a skewed graph one of them
loops over the neighbour lists of the low-degree endpoints and the other
over those of the hubs. The candidates are the model's top plans and their
mirrors, each with and without inclusion-exclusion (an inclusion-exclusion
plan gives up the bitmap subtree, which dense patterns need); the fastest on
the sample wins. A candidate whose sample outlives a cycle limit is dropped.
A short sample launch is paced by its slowest task rather than by
throughput, so the candidates are compared by the launch's busy warp cycles
(each warp's cycles until it found no work left, summed), which measure the
sample's total work however unevenly it spread; ``project_s`` turns them
into a projected time for the whole count.
"""

import ctypes
import itertools
import json
import os

from . import _native as N

DEFAULT_SPACE = {
    "blocks_per_sm": [2, 3, 4],
    "lane_work": [64, 192, 512],
    "core": [True, False],
    "chunk": [0, 4],
    "split": [1, 8],
}


def _key(graph, sched, idx, device):
    st = graph.stats(with_triangles=False)
    order, res, _ = sched.get(idx)
    return json.dumps({"device": device, "n": st["n"], "m": st["m"], "max_deg": st["max_deg"],
                       "order": order, "res": res}, sort_keys=True)


def opts_for(cfg, **extra):
    flags = 0 if cfg.get("core", True) else N.GP_COUNT_NO_CORE
    return N.make_opts(blocks_per_sm=cfg["blocks_per_sm"], lane_work=cfg["lane_work"],
                       chunk=cfg["chunk"], split=cfg.get("split", 1), flags=flags | extra.pop("flags", 0),
                       **extra)


def sample_ranges(nnz, windows, width, seed=0):
    """Stratified task windows: one window of `width` tasks at a seeded
    offset inside each of `windows` equal slices of the task space (every
    task equally likely to be sampled)."""
    if nnz <= windows * width:
        return [(0, nnz)]
    step = nnz // windows
    out = []
    for i in range(windows):
        off = int(((i * 0x9E3779B97F4A7C15 + seed) >> 7) % max(1, step - width))
        out.append((i * step + off, min(nnz, i * step + off + width)))
    return out


def time_config(graph, sched, idx, cfg, ranges, reps=2, stream=None):
    ms = ctypes.c_float()
    best = None
    counts = None
    import numpy as np
    for _ in range(reps):
        o = opts_for(cfg, kernel_ms=ctypes.pointer(ms))
        raw = np.zeros(2 * len(ranges), dtype=np.uint64)
        st, out, nxt = N.gp_count_batch_ranges([graph] * len(ranges), [sched] * len(ranges),
                                               [idx] * len(ranges), [a for a, _ in ranges],
                                               [b for _, b in ranges], o, stream=stream, raw=raw)
        if st != N.GP_OK:
            raise RuntimeError("sample count did not complete")
        c = [int(raw[2 * j]) | (int(raw[2 * j + 1]) << 64) for j in range(len(ranges))]
        if counts is not None and c != counts:
            raise AssertionError("autotuner sample counts differ between runs")
        counts = c
        best = ms.value if best is None else min(best, ms.value)
    return best, counts


def tune(graph, sched, idx=0, space=None, windows=64, width=2048, cache_path=None, stream=None,
         device=None):
    """Return (best configuration, table of (configuration, ms)). Every
    configuration must produce the same sample counts; a mismatch raises."""
    space = space or DEFAULT_SPACE
    if device is None:
        try:
            import torch
            device = torch.cuda.get_device_name()
        except Exception:
            device = "cuda"
    key = _key(graph, sched, idx, device)
    cache = {}
    if cache_path and os.path.exists(cache_path):
        with open(cache_path) as f:
            cache = json.load(f)
        if key in cache:
            return cache[key]["best"], cache[key]["table"]
    nnz = graph.device_csr()[2]
    ranges = sample_ranges(nnz, windows, width)
    names = list(space)
    table, ref = [], None
    for values in itertools.product(*(space[k] for k in names)):
        cfg = dict(zip(names, values))
        ms, counts = time_config(graph, sched, idx, cfg, ranges, stream=stream)
        if ref is None:
            ref = counts
        elif counts != ref:
            raise AssertionError(f"configuration {cfg} changed the sample counts")
        table.append((cfg, ms))
    best = min(table, key=lambda r: r[1])[0]
    if cache_path:
        cache[key] = {"best": best, "table": table}
        tmp = cache_path + ".tmp"
        with open(tmp, "w") as f:
            json.dump(cache, f)
        os.replace(tmp, cache_path)
    return best, table


def project_s(busy, done, total, clock_hz=2.07e9):
    """Projected time of a whole count from a sample launch: busy warp
    cycles x (all tasks / sampled tasks) / (warps x clock), i.e. the
    sample's total work spread evenly over the full launch's warps."""
    cycles, warps = busy
    if done <= 0 or warps <= 0:
        return None
    return cycles * (total / done) / (warps * clock_hz)


def plan_candidates(pattern, graph, top_k=3, stream=None):
    """(order, restrictions) of the model's top_k plans and of their mirror
    images (every restriction reversed: a valid set of the same model cost),
    without repeats, the model's first plan first."""
    top = N.gp_schedule(pattern, graph, top_k=top_k, stream=stream)
    out = []
    for i in range(len(top)):
        order, res, _ = top.get(i)
        for r in (tuple(res), tuple((b, a) for a, b in res)):
            if (order, r) not in out:
                out.append((order, r))
    return out


def choose_plan(graph, adj, top_k=3, iep=True, windows=256, width=64, item_s=2.0, cache_path=None,
                stream=None, device=None):
    """Time every candidate plan of the pattern `adj` on one stratified task
    sample and return (schedules handle of the fastest, table of
    (order, restrictions, inclusion-exclusion loops, ms or None)). Results
    are cached per (device, graph statistics, pattern)."""
    import numpy as np
    if device is None:
        try:
            import torch
            device = torch.cuda.get_device_name()
        except Exception:
            device = "cuda"
    adj = np.ascontiguousarray(adj, dtype=np.uint8)
    pattern = N.gp_pattern_create(adj)
    st = graph.stats(with_triangles=False)
    key = json.dumps({"device": device, "n": st["n"], "m": st["m"], "max_deg": st["max_deg"],
                      "pattern": adj.tolist(), "top_k": top_k, "iep": iep, "windows": windows, "width": width,
                      "choose_plan": 3}, sort_keys=True)
    cache = {}
    if cache_path and os.path.exists(cache_path):
        with open(cache_path) as f:
            cache = json.load(f)
    if key in cache:
        order, res, use_iep = cache[key]["best"]
        sched = N.gp_schedule_explicit(pattern, order, [tuple(r) for r in res])
        if use_iep:
            sched.set_iep(True)
        return sched, cache[key]["table"]
    nnz = graph.device_csr()[2]
    ranges = sample_ranges(nnz, windows, width)
    ms = ctypes.c_float()
    table, best = [], None
    cands = []
    for order, res in plan_candidates(pattern, graph, top_k, stream):
        cands.append((order, res, False))
        if iep:
            cands.append((order, res, True))
    for order, res, use_iep in cands:
        sched = N.gp_schedule_explicit(pattern, order, list(res))
        if use_iep and sched.set_iep(True) == 0:
            continue                                    # inclusion-exclusion does not apply
        raw = np.zeros(2 * len(ranges), dtype=np.uint64)
        busy = (ctypes.c_uint64 * 2)()
        o = N.make_opts(kernel_ms=ctypes.pointer(ms), task_cycles=int(item_s * 1.9e9),
                        budget_cycles=int(4 * item_s * 1.9e9),
                        busy_cycles=ctypes.cast(busy, ctypes.POINTER(ctypes.c_uint64)))
        status, _, nxt = N.gp_count_batch_ranges([graph] * len(ranges), [sched] * len(ranges),
                                                 [0] * len(ranges), [a for a, _ in ranges],
                                                 [b for _, b in ranges], o, stream=stream, raw=raw)
        done = sum(b - a for a, b in ranges)
        t = project_s((busy[0], busy[1]), done, nnz) if status == N.GP_OK else None   # stopped: dropped
        table.append((list(order), [list(r) for r in res], sched.iep(0)[0], t))
        if t is not None and (best is None or t < best[0]):
            best = (t, sched, (list(order), [list(r) for r in res], use_iep))
    if best is None:                                    # nothing finished the sample: the model's pick
        order, res = plan_candidates(pattern, graph, 1, stream)[0]
        sched = N.gp_schedule_explicit(pattern, order, list(res))
        best = (None, sched, (list(order), [list(r) for r in res], False))
    if cache_path:
        cache[key] = {"best": best[2], "table": table}
        tmp = cache_path + ".tmp"
        with open(tmp, "w") as f:
            json.dump(cache, f)
        os.replace(tmp, cache_path)
    return best[1], table
