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


def sample_ranges(nnz, windows, width):
    """Evenly spaced task windows covering the whole task space."""
    if nnz <= windows * width:
        return [(0, nnz)]
    step = nnz // windows
    return [(i * step, min(nnz, i * step + width)) for i in range(windows)]


def time_config(graph, sched, idx, cfg, ranges, reps=2, stream=None):
    ms = ctypes.c_float()
    best = None
    counts = None
    for _ in range(reps):
        o = opts_for(cfg, kernel_ms=ctypes.pointer(ms))
        st, out, nxt = N.gp_count_batch_ranges([graph] * len(ranges), [sched] * len(ranges),
                                               [idx] * len(ranges), [a for a, _ in ranges],
                                               [b for _, b in ranges], o, stream=stream)
        if st != N.GP_OK:
            raise RuntimeError("sample count did not complete")
        c = [int(x) for x in out]
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
