#!/usr/bin/env python
"""Benchmark: pattern-count time on a device-resident synthetic graph.

One step counts every pattern of the workload once with the plan chosen
among the performance model's top plans and their mirror images by a task
sample (--model-plan: the model's first); graph build and planning are
excluded, as in the paper's evaluation, and appear in the end-to-end number
instead.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload rmat20]
  python bench.py --impl reference ...   # the CPU oracle on a bounded sample

With --gpus N > 1 (launched by torch.distributed.run) every rank holds a
replica of the graph and counts a contiguous share of every pattern's edge
tasks; the per-rank partial counts are summed across ranks once per step.
"""

import argparse
import ctypes
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2009_10955_gb300.shard import (allreduce_counts, graph_row_ptr, rank_tasks,  # noqa: E402,F401
                                          shard_range, shard_roots)
from synth import named_pattern, workload_edges  # noqa: E402

WORKLOADS = {
    # R-MAT scale 20, edge factor 16, a/b/c/d .57/.19/.19/.05, seed 2; the
    # House and the 6-cycle run outside the timed step, each as one whole
    # count under a device budget (the 6-cycle needs hours: no
    # inclusion-exclusion applies, as no two non-adjacent vertices leave a
    # connected rest)
    "rmat20": {"graph": "rmat20", "patterns": ["triangle", "k4", "k5"], "projected": ["house", "c6"]},
    # House on G(2000, 20000), seed 1
    "er2000": {"graph": "er2000", "patterns": ["house"], "projected": []},
    # Chung-Lu 4M vertices, 35M pairs, exponent 2.1, max expected degree 20K,
    # seed 3
    "cl4m": {"graph": "cl4m", "patterns": ["k6e"], "projected": ["c6chord", "grid3x2"]},
}

L2_FLUSH_BYTES = 512 << 20          # larger than the 129 MB L2

# knobs the bench lets the autotuner choose per pattern
BENCH_TUNE_SPACE = {"blocks_per_sm": [3, 4], "lane_work": [96, 192, 512], "core": [True],
                    "chunk": [0], "split": [1, 8]}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="rmat20", choices=sorted(WORKLOADS))
    ap.add_argument("--patterns", default=None, help="comma list overriding the workload's patterns")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--tune", action="store_true",
                    help="let the autotuner pick launch knobs per pattern (default: library defaults, which "
                         "measured faster on the full count than the tuner's task-sample choice)")
    ap.add_argument("--model-plan", action="store_true",
                    help="count with the plan the performance model ranks first (default: the fastest of the "
                         "model's top three plans and their mirror images on a task sample, autotune.choose_plan)")
    ap.add_argument("--no-iep", action="store_true",
                    help="plain enumeration only (default: inclusion-exclusion for the innermost loops where a "
                         "plan qualifies, Section IV-D)")
    ap.add_argument("--cpu-seconds", type=float, default=20.0, help="CPU-baseline sample budget")
    ap.add_argument("--project-limit-s", type=float, default=120.0,
                    help="patterns outside the step: the device budget of their whole count")
    ap.add_argument("--batched-graph", default="rmat20",
                    help="graph of the batched comparison (64 random patterns x top-3 plans; '' to skip)")
    ap.add_argument("--mode", default="count",
                    choices=["count", "serve", "model", "case", "iep", "directed", "plan"],
                    help="serve: the continuous-batching sweep; model: performance-model accuracy; "
                         "case: one untimed count of each pattern on --graph (for profiler captures); "
                         "plan: host planning time of every named pattern (no GPU needed)")
    ap.add_argument("--graph", default="rmat16", help="synthetic graph of --mode case")
    ap.add_argument("--case-range", default="0,1",
                    help="--mode case: the fraction range [a, b) of the edge tasks to count")
    ap.add_argument("--iep-cases", default="rmat14/star5,rmat14/star6,rmat16/star5,rmat16/star6,"
                    "rmat14/three_ears,rmat16/three_ears,rmat14/house,rmat16/house,rmat20/house,cl1000000/k6e",
                    help="graph/pattern pairs of --mode iep")
    ap.add_argument("--model-graph", default="rmat20")
    ap.add_argument("--model-patterns", default="triangle,k4,house,k5")
    ap.add_argument("--serve-scales", default="14,15,16,17,18,19,20,22")
    ap.add_argument("--serve-rates", default="10,30,100,300,1000")
    ap.add_argument("--serve-requests", type=int, default=200)
    ap.add_argument("--serve-deadline", type=float, default=2.0)
    ap.add_argument("--serve-slice-ms", type=float, default=5.0)
    ap.add_argument("--serve-mem-gb", type=float, default=2.0,
                    help="device memory budget for the intermediate-set scratch of a time slice")
    return ap.parse_args()


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


ALU_LANES_PER_SMSP = 16     # integer/logic (ALU pipe) lanes per SM sub-partition per cycle
SMSP_PER_SM = 4


def alu_peak_gops(nsm):
    """Integer ALU peak in 32-bit lane operations per second (Gop/s): SMs x 4
    sub-partitions x 16 ALU lanes x the maximum SM clock (MEASURED_PEAKS.json's
    sm_max_mhz, else the GB300's 2070 MHz)."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            mhz = float(json.load(f)["sm_max_mhz"])
        src = "measured sm_max_mhz"
    except Exception:
        mhz, src = 2070.0, "nominal 2070 MHz"
    return nsm * SMSP_PER_SM * ALU_LANES_PER_SMSP * mhz * 1e6 / 1e9, (
        f"{nsm} SMs x {SMSP_PER_SM} SMSPs x {ALU_LANES_PER_SMSP} ALU lanes x {mhz:.0f} MHz ({src})")


# ----------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi sampling of SM clock and throttle reasons during timing."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid):
        self.rows = []
        self.proc = None
        self.uuid = uuid
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", uuid, f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) == 8:
                self.rows.append(parts)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = self.rows
        note = None
        if not rows:
            # timed region shorter than the 200 ms sampling period: one query
            # right after it, while the clocks still reflect the load
            try:
                out = subprocess.run(["nvidia-smi", "-i", self.uuid, f"--query-gpu={self.FIELDS}",
                                      "--format=csv,noheader,nounits"], capture_output=True, text=True,
                                     timeout=10).stdout
                rows = [[x.strip() for x in line.split(",")] for line in out.splitlines()]
                rows = [r for r in rows if len(r) == 8]
                note = "timed region shorter than the sampling period; sampled right after it"
            except Exception:
                rows = []
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[0]) for r in rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[4 + i].lower() == "active"})
        out = {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
               "reasons": reasons, "samples": len(rows)}
        if note:
            out["note"] = note
        return out


# -------------------------------------------------------------- CPU baseline

def _oracle_worker(n, row_ptr, col, name, sets, threads, q):
    """Child process: time the oracle on the given root sets (begin, end,
    stride) of the degree-ordered graph (the oracle's CSR, built once by the
    parent), one set after another."""
    import oracle
    g = oracle.Csr(n, row_ptr, col)
    q.put(("ready", 0, 0.0))
    adj = named_pattern(name)
    for b, e, st in sets:
        t = time.time()
        oracle.count_maps(adj, g, root_begin=int(b), root_end=int(e), root_stride=int(st), threads=threads)
        q.put(("set", len(range(int(b), int(e), int(st))), time.time() - t))


def degree_strata(n, src, dst):
    """Root ranges [a, b) of the degree-ordered graph holding the vertices of
    degree in [2^i, 2^(i+1)) (degree order makes each stratum contiguous)."""
    # degrees of the simple graph: loops and duplicate pairs dropped
    a, b = np.minimum(src, dst).astype(np.int64), np.maximum(src, dst).astype(np.int64)
    keep = a != b
    key = np.unique(a[keep] * n + b[keep])
    deg = np.bincount(np.concatenate([key // n, key % n]), minlength=n)
    d = np.sort(deg)[::-1]
    out, start = [], 0
    while start < n and d[start] > 0:
        top = int(d[start])
        lo_deg = 1 << (top.bit_length() - 1)
        end = start + int(np.searchsorted(-d[start:], -lo_deg, side="right"))
        out.append((start, end, lo_deg))
        start = end
    return out


def cpu_baseline(n, src, dst, patterns, budget_s, seed=12345, per_set=64):
    """The oracle (plain unrestricted enumeration, all host cores) on a
    degree-stratified sample of root vertices, scaled to the whole graph.
    The roots are split into strata of degree [2^i, 2^(i+1)) (contiguous in
    the degree order); from every stratum one set of up to `per_set` evenly
    spaced roots (seeded offset) is timed to completion, lowest degrees
    first, each pattern with an equal share of the budget. A stratum's time
    is its set's time x stratum size / set size. Sets not reached, or cut at
    the budget (counted with the time they had used), make the estimate a
    lower bound, which is flagged. Both benchmark arms call this with the
    same seed, so they time the same root sets."""
    import multiprocessing as mp
    import queue as qmod
    import oracle
    threads = os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    rng = np.random.default_rng(seed)
    og, _ = oracle.degree_relabel(oracle.build_csr(n, src, dst))
    strata = degree_strata(n, src, dst)[::-1]       # lowest degrees first
    sets = []
    for a, b, _ in strata:
        st = max(1, (b - a) // per_set)
        off = int(rng.integers(0, st))
        sets.append((a + off, b, st))
    per = budget_s / max(1, len(patterns))
    est, parts, lower = 0.0, [], False
    for name in patterns:
        q = ctx.Queue()
        proc = ctx.Process(target=_oracle_worker, args=(n, og.row_ptr, og.col, name, sets, threads, q), daemon=True)
        proc.start()
        try:
            q.get(timeout=900)                       # CSR built; the clock starts now
        except qmod.Empty:
            proc.terminate()
            raise RuntimeError("oracle CSR build did not finish")
        t0 = time.time()
        t_last = t0
        pat_est, done = 0.0, 0
        for (a, b, _), (sb, se, st) in zip(strata, sets):
            left = per - (time.time() - t0)
            try:
                if left <= 0:
                    raise qmod.Empty
                _, r, dt = q.get(timeout=left)
                t_last = time.time()
                pat_est += dt * (b - a) / max(r, 1)
                done += 1
            except qmod.Empty:
                # the set is cut: the time it had used stands for its whole
                # stratum, and the strata after it add nothing
                lower = True
                pat_est += (time.time() - t_last) * (b - a) / max(1, len(range(sb, se, st)))
                break
        if proc.is_alive():
            proc.terminate()
            proc.join(timeout=10)
        est += pat_est
        parts.append(f"{name}: {done} of {len(strata)} degree strata timed in {time.time() - t0:.1f} s")
    return {"value": est, "unit": "s", "cores": threads, "kind": "oracle",
            "sample": "; ".join(parts) + f"; per stratum of degree [2^i, 2^(i+1)) one set of up to {per_set} "
                      "evenly spaced roots, estimate = sum over strata of set time x stratum size / set size",
            "lower_bound": lower}


# ------------------------------------------------------- multi-rank helpers
# the root partition and the exact 128-bit all-reduce live in the package
# (paper_2009_10955_gb300/shard.py); the bench re-exports them

# ------------------------------------------------------------------ GPU arm

def _code_only(text):
    """C/C++/CUDA source without comments and with whitespace runs collapsed:
    what the compiler sees, so that editing a comment keeps a recorded
    measurement valid."""
    out, i, n = [], 0, len(text)
    while i < n:
        c = text[i]
        if c == '"' or c == "'":                       # literal: copy through its end
            j = i + 1
            while j < n and text[j] != c:
                j += 2 if text[j] == "\\" else 1
            out.append(text[i:j + 1])
            i = j + 1
        elif text.startswith("//", i):
            j = text.find("\n", i)
            i = n if j < 0 else j
        elif text.startswith("/*", i):
            j = text.find("*/", i + 2)
            i = n if j < 0 else j + 2
            out.append(" ")
        else:
            out.append(c)
            i += 1
    return " ".join("".join(out).split())


def source_hash():
    """Hash of the count kernel's code and of the planner that compiles its
    plans, comments excluded."""
    h = hashlib.sha256()
    for f in ("count.cu", "plan.h", "planner.cpp"):
        with open(os.path.join(ROOT, "paper_2009_10955_gb300", "csrc", f), encoding="utf-8") as fh:
            h.update(_code_only(fh.read()).encode())
    return h.hexdigest()[:16]


def recorded_traffic(workload):
    """Per-launch DRAM bytes of the count kernel for each pattern of a
    workload, from a committed ncu summary, used only while the kernel source
    is unchanged since the capture ({} otherwise)."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            t = json.load(f)
        e = t.get(workload)
        if e and e.get("source_hash") == source_hash():
            return dict(e.get("dram_bytes_per_launch") or e.get("per_launch") or {})
    except Exception:
        pass
    return {}


_T0 = time.time()


def phase(name):
    """Progress line on stderr: seconds since start and the phase begun."""
    print(f"[bench {time.time() - _T0:7.1f} s] {name}", file=sys.stderr, flush=True)


def workload_config(workload, graph, n, m_undirected, max_deg, patterns):
    """The `config` of both benchmark arms: what the workload is (graph,
    its size, the patterns of one step) and how L2 is treated between timed
    GPU counts. Run results and the method's choices go elsewhere in the
    line, so the two arms report one identical config."""
    return {"workload": workload, "graph": graph, "n": int(n), "m_undirected": int(m_undirected),
            "max_deg": int(max_deg), "patterns": list(patterns),
            "l2": "GPU counts: L2 flushed (512 MB write) before every count"}


def gpu_arm(a, rank, world):
    import torch
    import torch.distributed as dist
    from paper_2009_10955_gb300 import native
    N = native()
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream(dev)
    wl = WORKLOADS[a.workload]
    pats = a.patterns.split(",") if a.patterns else wl["patterns"]
    n, src, dst = workload_edges(wl["graph"])

    phase("graph build")
    t = time.time()
    g = N.gp_graph_create_edges(src, dst, n, N.GP_DEGREE_ORDER, stream=stream)
    torch.cuda.synchronize()
    build_s = time.time() - t
    st = g.stats(stream=stream)
    nnz = g.device_csr()[2]
    def make_plan(p, graph):
        s = N.gp_schedule(N.gp_pattern_create(named_pattern(p)), graph, top_k=1, stream=stream)
        if not a.no_iep:
            s.set_iep(True)
        return s

    phase("plans")
    plans, plan_s, plan_table = {}, {}, {}
    cache = os.path.join(ROOT, "paper_2009_10955_gb300", "_build", "tune_cache.json")
    for p in pats:
        t = time.time()
        if a.model_plan:
            plans[p] = make_plan(p, g)
        else:
            from paper_2009_10955_gb300 import autotune
            plans[p], plan_table[p] = autotune.choose_plan(g, named_pattern(p), top_k=3, iep=not a.no_iep,
                                                           cache_path=cache, stream=stream)
        plan_s[p] = time.time() - t
    model_pick = {p: autotune_first(N, g, p, stream) for p in pats}
    # this rank's share of every pattern's edge tasks: whole roots, balanced
    # by the sum of squared degrees
    if world > 1:
        lo, hi = rank_tasks(graph_row_ptr(g), rank, world)
    else:
        lo, hi = 0, nnz

    # launch knobs per pattern from the autotuner (untimed, cached like plans)
    tuned, tune_s = {}, {}
    if a.tune:                               # the tuner samples task ranges
        from paper_2009_10955_gb300 import autotune
        for p in pats:
            t = time.time()
            tuned[p], _ = autotune.tune(g, plans[p], 0, space=BENCH_TUNE_SPACE, windows=64, width=1024,
                                        cache_path=cache, stream=stream)
            tune_s[p] = time.time() - t
    def knobs(p, **kw):
        if p in tuned:
            from paper_2009_10955_gb300 import autotune
            return autotune.opts_for(tuned[p], **kw)
        return N.make_opts(**kw)

    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    ms = ctypes.c_float()

    raw_buf = (ctypes.c_uint64 * 2)()

    def count(p, timed):
        """One timed count; returns the undivided total of this rank's tasks
        (the count for plain plans), the call's and the kernel's ms."""
        if hi <= lo:                                       # an empty share (task_end 0 would mean all)
            return 0, 0.0, 0.0
        flush.fill_(1)                                     # evict the graph from L2
        o = knobs(p, task_begin=lo, task_end=hi, kernel_ms=ctypes.pointer(ms),
                  raw_total=ctypes.cast(raw_buf, ctypes.POINTER(ctypes.c_uint64)))
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        status, c = N.gp_count(g, plans[p], 0, o, stream=stream)
        e1.record(stream)
        e1.synchronize()
        if status != N.GP_OK:
            raise RuntimeError(f"count of {p} returned status {status}")
        return int(raw_buf[0]) | (int(raw_buf[1]) << 64), e0.elapsed_time(e1), ms.value

    phase("instrumented counts")
    # algorithmic work per pattern (instrumented kernel on the same paths as
    # the timed launch, untimed): list-path bytes and bitmap word operations
    algo, algo_ops = {}, {}
    for p in pats:
        b, ops = ctypes.c_uint64(), ctypes.c_uint64()
        raw = (ctypes.c_uint64 * 2)()
        o = knobs(p, task_begin=lo, task_end=hi, flags=N.GP_COUNT_STATS, algo_bytes=ctypes.pointer(b),
                  algo_ops=ctypes.pointer(ops), raw_total=ctypes.cast(raw, ctypes.POINTER(ctypes.c_uint64)))
        N.gp_count(g, plans[p], 0, o, stream=stream)
        algo[p], algo_ops[p] = b.value, ops.value

    phase("warm-up and timed steps")
    for _ in range(a.warmup):
        for p in pats:
            count(p, False)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    uuid = str(torch.cuda.get_device_properties(dev).uuid)
    clocks = ClockSampler(uuid if uuid.startswith("GPU-") else "GPU-" + uuid)
    N.gp_take_launch_count()
    step_ms, kern_ms, counts = [], {p: [] for p in pats}, {}
    for _ in range(a.steps):
        tot = 0.0
        for p in pats:
            c, call_ms, kms = count(p, True)
            tot += call_ms
            kern_ms[p].append(kms)
            counts[p] = c
        step_ms.append(tot)
    launches = N.gp_take_launch_count()
    torch.cuda.synchronize()
    clk = clocks.stop()

    # sum partial totals over ranks (the one exchange of the sharded path),
    # then divide inclusion-exclusion totals by their plan's divisor
    if world > 1:
        summed = allreduce_counts([counts[p] for p in pats], device=dev)
        counts = dict(zip(pats, summed))
        t_local = torch.tensor([statistics.mean(step_ms)], device=dev)
        dist.all_reduce(t_local, op=dist.ReduceOp.MAX)
        mean_step = float(t_local[0])
    else:
        mean_step = statistics.mean(step_ms)
    for p in pats:
        div = plans[p].iep(0)[1]
        if counts[p] % div:
            raise RuntimeError(f"{p}: total {counts[p]} is not a multiple of its divisor {div}")
        counts[p] //= div

    phase("end to end")
    # end to end through the C ABI with host buffers: graph from host pairs,
    # planning, counts and 8-byte results back
    e2e_ms = []
    # the step's inputs sit in pinned host memory, as a serving process keeps them
    src_h = torch.from_numpy(np.ascontiguousarray(src, dtype=np.int32)).pin_memory().numpy()
    dst_h = torch.from_numpy(np.ascontiguousarray(dst, dtype=np.int32)).pin_memory().numpy()
    for _ in range(max(1, min(3, a.steps))):
        torch.cuda.synchronize()
        t = time.time()
        g2 = N.gp_graph_create_edges(src_h, dst_h, n, N.GP_DEGREE_ORDER, stream=stream)
        for p in pats:
            order, res, _ = plans[p].get(0)
            N.gp_schedule(N.gp_pattern_create(named_pattern(p)), g2, top_k=1, stream=stream)   # the model
            s2 = N.gp_schedule_explicit(N.gp_pattern_create(named_pattern(p)), order, res)
            if not a.no_iep:
                s2.set_iep(True)
            N.gp_count(g2, s2, 0, knobs(p, task_begin=lo, task_end=hi,
                                        raw_total=ctypes.cast(raw_buf, ctypes.POINTER(ctypes.c_uint64))),
                       stream=stream)
        torch.cuda.synchronize()
        e2e_ms.append((time.time() - t) * 1000.0)
        del g2

    # patterns of the workload that no bench-sized step can count: a rate
    # from a stratified task sample and the projected time (labelled)
    projected = {}
    phase("patterns outside the step")
    if world == 1 and not a.patterns:
        for p in wl.get("projected", []):
            if a.model_plan:
                sp = make_plan(p, g)
            else:
                from paper_2009_10955_gb300 import autotune
                sp, _ = autotune.choose_plan(g, named_pattern(p), top_k=3, iep=not a.no_iep,
                                             cache_path=cache, stream=stream)
            rec = budgeted_count(N, g, sp, stream, a.project_limit_s)
            rec.update({"order": sp.get(0)[0], "restrictions": sp.get(0)[1], "iep_loops": sp.iep(0)[0]})
            if "count" not in rec:
                rec["sample"] = timed_or_projected(N, g, sp, stream, limit_s=0.0, sample_s=10.0)
            projected[p] = rec

    batched = None
    phase("batched comparison")
    if a.batched_graph and world == 1:
        batched = batched_compare(N, stream, a.batched_graph)

    hbm, peak_kind = peaks()
    # L2 copy bandwidth measured in this run: 2 x 24 MB buffers (48 MB
    # working set, inside the 129 MB L2), read + write bytes per copy
    xa = torch.empty(24 << 20, dtype=torch.uint8, device=dev)
    xb = torch.empty_like(xa)
    for _ in range(5):
        xb.copy_(xa)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 200
    e0.record(stream)
    for _ in range(reps):
        xb.copy_(xa)
    e1.record(stream)
    e1.synchronize()
    l2_gbs = 2 * xa.numel() * reps / (e0.elapsed_time(e1) / 1000.0) / 1e9
    del xa, xb
    mean_kern = {p: statistics.mean(v) for p, v in kern_ms.items()}
    kern_total_ms = sum(mean_kern.values())
    traffic = recorded_traffic(a.workload)
    nsm = torch.cuda.get_device_properties(dev).multi_processor_count
    alu_peak, alu_src = alu_peak_gops(nsm)
    # per launch: list-path bytes against the HBM copy peak, bitmap word
    # operations against the integer ALU peak; the bound is the larger share
    per = {}
    for p in pats:
        t = mean_kern[p] / 1000.0
        gbs = algo[p] / t / 1e9 if t > 0 else 0.0
        gops = algo_ops[p] / t / 1e9 if t > 0 else 0.0
        per[p] = {"launch_s": t, "share_of_step": mean_kern[p] / kern_total_ms if kern_total_ms else None,
                  "list_bytes": algo[p], "list_gbs": gbs, "hbm_frac": gbs / hbm,
                  "bitmap_ops": algo_ops[p], "bitmap_gops": gops, "alu_frac": gops / alu_peak,
                  "dram_bytes": traffic.get(p)}
        per[p]["bound"] = "alu" if per[p]["alu_frac"] > per[p]["hbm_frac"] else "hbm"
    dom = max(pats, key=lambda p: mean_kern[p])
    d = per[dom]
    if d["bound"] == "alu":
        roof = {"bound": "alu", "achieved": d["bitmap_gops"], "peak": alu_peak, "unit": "Gop/s",
                "frac": d["alu_frac"], "peak_source": alu_src,
                "algorithmic_per_launch": d["bitmap_ops"],
                "algorithmic_unit": "32-bit word operations of the bitmap subtree (AND, POPC, scatter) and "
                                    "candidates taken from its sets, tallied by the instrumented build"}
    else:
        roof = {"bound": "hbm", "achieved": d["list_gbs"], "peak": hbm, "unit": "GB/s", "frac": d["hbm_frac"],
                "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured"
                else "fallback 6.8 TB/s",
                "algorithmic_per_launch": d["list_bytes"],
                "algorithmic_unit": "bytes of the list intersections executed (merge or search, whichever is "
                                    "cheaper), stored elements and iterated candidates"}
    roof.update({"traffic": d["dram_bytes"], "kernel": f"k_count ({dom} launch)", "launch_s": d["launch_s"],
                 "share_of_step": d["share_of_step"], "l2_peak_gbs": l2_gbs,
                 "per_pattern": per,
                 "traffic_source": "profiles/traffic.json (ncu dram__bytes_read.sum + dram__bytes_write.sum "
                                   "per launch), null when the kernel changed since the capture"})
    out = {
        "metric": "pattern-count time (s)",
        "value": mean_step / 1000.0,
        "unit": "s",
        "n_gpus": world,
        "steps": a.steps,
        "warmup": a.warmup,
        "ms_per_step": mean_step,
        "higher_is_better": False,
        "scaling": "strong",
        "vs_baseline": None,
        "dtype": "int32",
        "data": "synthetic",
        "config": workload_config(a.workload, wl["graph"], st["n"], st["m"], st["max_deg"], pats),
        "results": {
            "counts": {p: counts[p] for p in pats},
            "per_pattern_s": {p: mean_kern[p] / 1000.0 for p in pats},
            "plans": {p: {"order": plans[p].get(0)[0], "restrictions": plans[p].get(0)[1],
                          "iep_loops": plans[p].iep(0)[0], "iep_divisor": plans[p].iep(0)[1],
                          "model_first": tuple(plans[p].get(0)[:2]) == model_pick[p]} for p in pats},
            "plan_choice": ("model's first plan" if a.model_plan else
                            "fastest on a 256 x 64-task sample of the model's top 3 plans and their mirror "
                            "images (autotune.choose_plan), untimed"),
            "plan_candidates": plan_table,
            "graph_build_s": build_s,
            "plan_s": plan_s,
            "tuned": tuned,
            "tune_s": tune_s,
        },
        "method": {"step": "one count of each pattern, device-resident graph",
                   "parallelism": f"edge tasks sharded over {world} GPU(s)"},
        "e2e": {"value": statistics.mean(e2e_ms) / 1000.0, "unit": "s",
                "h2d_bytes_per_step": int(src.nbytes + dst.nbytes),
                "d2h_bytes_per_step": 16 * len(pats),
                "includes": "graph build from host pairs in pinned memory, the performance model's ranking, "
                            "the chosen plan (cached choice, gp_schedule_explicit), counts, 16-byte totals to "
                            "host"},
        "gpu_launches": launches // max(1, a.steps),
        "roofline": roof,
        "clocks": clk,
        "batched": batched,
        "outside_step": projected,
    }
    return out, (n, src, dst, pats)


def autotune_first(N, g, p, stream):
    """(order, restrictions) of the plan the performance model ranks first."""
    return tuple(N.gp_schedule(N.gp_pattern_create(named_pattern(p)), g, top_k=1, stream=stream).get(0)[:2])


def batched_compare(N, stream, graph_name="rmat20", npat=64, top_k=3, seed=64, job_limit_s=1.0, total_s=15.0):
    """64 random connected 3-6-vertex patterns (edge probability 0.5), each
    under its top-3 plans with inclusion-exclusion where it applies: one
    batched call for all jobs (one persistent launch per kernel build)
    against one launch per (pattern, plan) and one batched launch per
    pattern (its plans together), on `graph_name`. A pattern
    is left out (and listed) when a task sample projects its first plan above
    `job_limit_s`, or when the included patterns' projections (x the plans
    each has) already reach `total_s`. Undivided 128-bit totals are compared
    job by job; counts beyond 64 bits are reported as exact integers."""
    import torch
    from synth import random_pattern_set
    pats = random_pattern_set(npat, 3, 6, 0.5, seed)
    n, src, dst = workload_edges(graph_name)
    g = N.gp_graph_create_edges(src, dst, n, N.GP_DEGREE_ORDER, stream=stream)
    nnz = g.device_csr()[2]
    scheds, proj = [], []
    for adj in pats:
        s = N.gp_schedule(N.gp_pattern_create(adj), g, top_k=top_k, stream=stream)
        s.set_iep(True)
        scheds.append(s)
        wins = sample_windows(nnz, 256, 32, seed=1)
        raw = np.zeros(2 * len(wins), dtype=np.uint64)
        busy = (ctypes.c_uint64 * 2)()
        o = N.make_opts(budget_cycles=int(job_limit_s * 1.9e9), task_cycles=int(job_limit_s / 2 * 1.9e9),
                        busy_cycles=ctypes.cast(busy, ctypes.POINTER(ctypes.c_uint64)))
        st, _, nxt = N.gp_count_batch_ranges([g] * len(wins), [s] * len(wins), [0] * len(wins),
                                             [a for a, _ in wins], [b for _, b in wins], o, stream=stream, raw=raw)
        done = sum(int(x) - a for x, (a, _) in zip(nxt, wins) if int(x) >= 0)
        bad = st != N.GP_OK or any(int(x) < 0 for x in nxt)
        from paper_2009_10955_gb300.autotune import project_s
        proj.append(float("inf") if bad else project_s((busy[0], busy[1]), done, nnz))
    keep, left_out, acc = [], [], 0.0
    for i in sorted(range(npat), key=lambda i: proj[i]):
        cost = proj[i] * len(scheds[i])
        if proj[i] <= job_limit_s and acc + cost <= total_s:
            keep.append(i)
            acc += cost
        else:
            left_out.append({"pattern": i, "k": int(pats[i].shape[0]), "edges": int(pats[i].sum() // 2),
                             "projected_s": proj[i] if proj[i] != float("inf") else None})
    keep.sort()
    jobs = [(i, j) for i in keep for j in range(len(scheds[i]))]
    G, S, I = [g] * len(jobs), [scheds[i] for i, _ in jobs], [j for _, j in jobs]

    def timed(fn):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r = fn()
        e1.record(stream)
        e1.synchronize()
        return r, e0.elapsed_time(e1) / 1000.0

    raw_b = np.zeros(2 * len(jobs), dtype=np.uint64)
    N.gp_count_batch(G, S, I, stream=stream, raw=raw_b)                      # warm-up
    _, tb = timed(lambda: N.gp_count_batch(G, S, I, stream=stream, raw=raw_b))
    batched = [int(raw_b[2 * q]) | (int(raw_b[2 * q + 1]) << 64) for q in range(len(jobs))]
    single, ts = timed(lambda: [N.gp_count_raw(g, scheds[i], j, stream=stream)[1] for i, j in jobs])
    if batched != single:
        raise AssertionError("batched totals differ from single launches")
    # one launch per pattern: the pattern's plans batched together
    def per_pattern():
        for i in keep:
            n_i = len(scheds[i])
            N.gp_count_batch([g] * n_i, [scheds[i]] * n_i, list(range(n_i)), stream=stream,
                             raw=np.zeros(2 * n_i, dtype=np.uint64))
    _, tp = timed(per_pattern)
    counts = {}
    for (i, j), r in zip(jobs, batched):
        div = scheds[i].iep(j)[1]
        if r % div:
            raise AssertionError(f"pattern {i} plan {j}: total not a multiple of its divisor")
        c = r // div
        if counts.setdefault(i, c) != c:
            raise AssertionError(f"pattern {i}: plans disagree")
    over64 = sum(1 for c in counts.values() if c >> 64)
    return {"graph": graph_name, "patterns": npat, "patterns_counted": len(keep), "jobs": len(jobs),
            "left_out": left_out, "batched_s": tb, "per_plan_launches_s": ts, "per_pattern_launches_s": tp,
            "speedup_vs_per_plan": ts / tb, "speedup_vs_per_pattern": tp / tb, "counts_agree": True,
            "counts_beyond_64_bits": over64,
            "iep_jobs": sum(1 for i, j in jobs if scheds[i].iep(j)[0] > 0),
            "selection": f"patterns whose first plan projects <= {job_limit_s} s (busy warp cycles of a "
                         f"256 x 32-task sample) and finishes it, "
                         f"cheapest first, until the included jobs project {total_s} s"}


def serve_bench(N, stream, scales, rates, per_rate, deadline_s, slice_ms, mem_budget=None, seed=777):
    """Continuous-batching server over several device-resident R-MAT graphs
    (scale s, edge factor 16, seed 100 + s) under Poisson arrivals of random
    connected 3-6-vertex patterns (edge probability 0.5), admitted while the
    slice's intermediate-set scratch fits `mem_budget` bytes. Requests that
    need more than `deadline_s` of service are answered with a timeout.
    Latency runs from each request's scheduled arrival time."""
    from synth import random_pattern_set
    from synth.graphs import rmat_edges
    from paper_2009_10955_gb300.serve import Server, poisson_arrivals
    graphs = {}
    for sc in scales:
        src, dst = rmat_edges(sc, 16, 0.57, 0.19, 0.19, seed=100 + sc)
        graphs[f"rmat{sc}"] = N.gp_graph_create_edges(src, dst, 1 << sc, N.GP_DEGREE_ORDER, stream=stream)
    names = sorted(graphs)
    pats = random_pattern_set(64, 3, 6, 0.5, seed)
    rows = []
    for ri, rate in enumerate(rates):
        arr = poisson_arrivals(rate, per_rate, seed + ri)
        srv = Server(graphs, slice_ms=slice_ms, stream=stream, item_ms=20 * slice_ms, deadline_s=deadline_s,
                     mem_budget=mem_budget)
        t0 = time.perf_counter()
        reqs = []
        for i, at in enumerate(arr):
            delay = t0 + at - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            reqs.append(srv.submit(names[i % len(names)], pats[i % len(pats)], arrival=t0 + at))
        for r in reqs:
            r.done.wait(3600)
        srv.close()
        ok = [r for r in reqs if r.error is None]
        lat = sorted(r.latency for r in ok)
        span = max(r.finish for r in reqs) - t0
        rows.append({"rate": rate, "requests": len(reqs), "completed": len(ok),
                     "timeouts": sum(isinstance(r.error, TimeoutError) for r in reqs),
                     "errors": sum(r.error is not None and not isinstance(r.error, TimeoutError) for r in reqs),
                     "p50_s": lat[len(lat) // 2] if lat else None,
                     "p99_s": lat[min(len(lat) - 1, int(0.99 * len(lat)))] if lat else None,
                     "counts_per_s": len(ok) / span if span > 0 else None,
                     "slices": srv.slices, "admission_deferrals": srv.deferrals})
    return {"metric": "serving latency and throughput", "graphs": names, "slice_ms": slice_ms,
            "deadline_s": deadline_s, "mem_budget_bytes": mem_budget, "rows": rows}


def sample_windows(nnz, windows, width, seed):
    """Stratified task windows (one per equal slice of the task space, at a
    seeded offset): the autotuner's sampler."""
    from paper_2009_10955_gb300.autotune import sample_ranges
    return sample_ranges(nnz, windows, width, seed)


def budgeted_count(N, g, s, stream, limit_s):
    """The whole count with a device budget of limit_s: the count and its
    kernel time when it finishes; else how many edge tasks (in CSR order,
    high-degree roots first) the budget covered. A budget stops the launch
    between task grabs, so the kernel time can exceed it by the longest
    task in flight."""
    nnz = g.device_csr()[2]
    ms = ctypes.c_float()
    cur = ctypes.c_int64(0)
    try:
        st, raw = N.gp_count_raw(g, s, 0, stream=stream, kernel_ms=ctypes.pointer(ms),
                                 budget_cycles=int(limit_s * 1.9e9), task_cycles=int(limit_s / 2 * 1.9e9),
                                 resume_cursor=ctypes.pointer(cur))
    except N.GraphPiError as e:
        if e.status != N.GP_ERR_TIMEOUT:
            raise
        return {"kind": f"a single edge task outlived {limit_s / 2:.0f} s; count abandoned"}
    if st == N.GP_OK:
        return {"kind": "counted", "count": raw // s.iep(0)[1], "kernel_s": ms.value / 1e3}
    return {"kind": f"not finished within a {limit_s:.0f} s budget", "kernel_s": ms.value / 1e3,
            "tasks_done": cur.value, "tasks": nnz}


def timed_or_projected(N, g, s, stream, limit_s=30.0, windows=1024, width=64, seed=0, sample_s=20.0):
    """Whole count and kernel time when a stratified task sample projects it
    below limit_s; else the projection, labelled as such. The projection is
    the sample launch's busy warp cycles (each warp's cycles until it found
    no work left, summed: the sample's total work) x (tasks / sampled tasks)
    / (warps x clock), i.e. that work spread evenly over the full launch; a
    sample's own duration would instead be paced by its slowest task.
    Returns a dict."""
    from paper_2009_10955_gb300.autotune import project_s
    nnz = g.device_csr()[2]
    wins = sample_windows(nnz, windows, width, seed)
    ms = ctypes.c_float()
    raw = np.zeros(2 * len(wins), dtype=np.uint64)
    busy = (ctypes.c_uint64 * 2)()
    o = N.make_opts(kernel_ms=ctypes.pointer(ms), budget_cycles=int(sample_s * 1.9e9),
                    task_cycles=int(sample_s / 4 * 1.9e9),
                    busy_cycles=ctypes.cast(busy, ctypes.POINTER(ctypes.c_uint64)))
    st, _, nxt = N.gp_count_batch_ranges([g] * len(wins), [s] * len(wins), [0] * len(wins),
                                         [a for a, _ in wins], [b for _, b in wins], o, stream=stream, raw=raw)
    done = sum(int(x) - a for x, (a, _) in zip(nxt, wins) if int(x) >= 0)
    abandoned = sum(1 for x in nxt if int(x) < 0)
    proj = project_s((busy[0], busy[1]), done, nnz) or float("inf")
    rec = {"sample_tasks": done, "sample_s": ms.value / 1e3, "abandoned_windows": abandoned,
           "projected_s": proj}
    if proj < limit_s and abandoned == 0 and st == N.GP_OK:
        kms = ctypes.c_float()
        c = N.gp_count(g, s, 0, N.make_opts(kernel_ms=ctypes.pointer(kms)), stream=stream)[1]
        rec.update({"count": c, "kernel_s": kms.value / 1e3})
    return rec


def iep_bench(N, stream, cases, limit_s=30.0):
    """Inclusion-exclusion (Section IV-D) against plain enumeration on the
    same plan: for each (graph, pattern) the model's first plan is counted
    both ways (whole counts when feasible, else projections from a task
    sample, labelled), counts checked equal."""
    rows = []
    graphs = {}
    for gname, pname in cases:
        if gname not in graphs:
            n, src, dst = workload_edges(gname)
            graphs[gname] = N.gp_graph_create_edges(src, dst, n, N.GP_DEGREE_ORDER, stream=stream)
        g = graphs[gname]
        plain = N.gp_schedule(N.gp_pattern_create(named_pattern(pname)), g, top_k=1, stream=stream)
        iep = N.gp_schedule(N.gp_pattern_create(named_pattern(pname)), g, top_k=1, stream=stream)
        iep.set_iep(True)
        row = {"graph": gname, "pattern": pname, "plan": plain.get(0)[:2], "iep_loops": iep.iep(0)[0],
               "iep_divisor": iep.iep(0)[1],
               "plain": timed_or_projected(N, g, plain, stream, limit_s),
               "iep": timed_or_projected(N, g, iep, stream, limit_s)}
        a, b = row["plain"], row["iep"]
        if "count" in a and "count" in b and a["count"] != b["count"]:
            raise AssertionError(f"{gname}/{pname}: plain {a['count']} != inclusion-exclusion {b['count']}")
        ta = a.get("kernel_s", a["projected_s"])
        tb = b.get("kernel_s", b["projected_s"])
        row["speedup"] = ta / tb if tb > 0 else None
        row["speedup_kind"] = "measured" if "kernel_s" in a and "kernel_s" in b else "projected"
        rows.append(row)
        print(json.dumps(row, default=str), file=sys.stderr, flush=True)
    return {"metric": "inclusion-exclusion vs plain enumeration", "rows": rows}


DIRECTED_PATTERNS = {
    "cycle3": [(0, 1), (1, 2), (2, 0)],
    "feed_forward": [(0, 1), (0, 2), (1, 2)],
    "cycle4": [(0, 1), (1, 2), (2, 3), (3, 0)],
    "bifan": [(0, 2), (0, 3), (1, 2), (1, 3)],
}


def directed_bench(N, stream, scales=(12, 14), reps=3):
    """Directed patterns (the reading of an extension the paper names) on
    R-MAT graphs taken as digraphs (each sampled pair an arc src -> dst,
    loops and repeated arcs dropped): time of gp_dcount with the planner's
    configuration, best of `reps` synchronous calls after one warm-up."""
    from synth.graphs import rmat_edges
    rows = []
    for sc in scales:
        src, dst = rmat_edges(sc, 16, 0.57, 0.19, 0.19, seed=2)
        g = N.gp_dgraph_create(src, dst, 1 << sc, stream=stream)
        st = g.stats()
        for name, arcs in DIRECTED_PATTERNS.items():
            k = 1 + max(max(a, b) for a, b in arcs)
            adj = np.zeros((k, k), np.uint8)
            for a, b in arcs:
                adj[a, b] = 1
            p = N.gp_dpattern_create(adj)
            c = N.gp_dcount(g, p, stream=stream)
            best = None
            for _ in range(reps):
                t = time.perf_counter()
                c2 = N.gp_dcount(g, p, stream=stream)
                dt = time.perf_counter() - t
                best = dt if best is None else min(best, dt)
                if c2 != c:
                    raise AssertionError(f"{name} on rmat{sc}: counts differ between calls")
            rows.append({"graph": f"rmat{sc} (directed)", "n": st["n"], "arcs": st["narcs"], "pattern": name,
                         "count": c, "call_s": best})
            print(json.dumps(rows[-1]), file=sys.stderr, flush=True)
    return {"metric": "directed pattern count time (s)", "rows": rows,
            "timing": "wall time of the synchronous gp_dcount call (planning included), best of 3"}


def model_bench(N, stream, graph_name, patterns, max_configs=40, limit_s=5.0, iep=False):
    """Performance-model accuracy (the shape of the paper's Fig. 9, Fig. 10
    and Table II on a synthetic graph): every efficient schedule x
    restriction set (evenly subsampled beyond max_configs, the model's pick
    always included) is timed on one stratified task sample (256 windows of
    64 tasks; all configurations on the same windows), and counted whole
    when the sample projects it below limit_s (whole counts must agree). The
    model's pick is compared with the best configuration, and the spread of
    restriction sets under the picked schedule is reported."""
    n, src, dst = workload_edges(graph_name)
    g = N.gp_graph_create_edges(src, dst, n, N.GP_DEGREE_ORDER, stream=stream)
    st = g.stats(stream=stream)
    rows = []
    for name in patterns:
        p = N.gp_pattern_create(named_pattern(name))
        scheds, _ = p.schedules()
        sets = p.restriction_sets()
        pairs = [(sc, rs) for sc in scheds for rs in sets]
        step = max(1, len(pairs) // max_configs)
        pairs = pairs[::step]
        pick = N.gp_schedule(p, g, top_k=1, stream=stream).get(0)[:2]
        if pick not in pairs:
            pairs.append(pick)
        timed, count = [], None
        for sc, rs in pairs:
            one = N.gp_schedule_explicit(p, sc, rs)
            if iep:
                one.set_iep(True)
            rec = timed_or_projected(N, g, one, stream, limit_s=limit_s, sample_s=limit_s)
            if "count" in rec:
                if count is None:
                    count = rec["count"]
                elif rec["count"] != count:
                    raise AssertionError(f"{name}: configuration {sc} {rs} gave {rec['count']}, expected {count}")
            t = rec.get("kernel_s", rec["projected_s"])
            cost = N.gp_config_cost(p, sc, rs, st["n"], st["m"], st["tri_cnt"])
            timed.append((t, cost, sc, rs, "kernel_s" in rec))
        times = [x[0] for x in timed]
        best = min(times)
        pick_t = next(x[0] for x in timed if (x[2], x[3]) == pick)
        rc = np.argsort(np.argsort([x[1] for x in timed]))
        rt = np.argsort(np.argsort(times))
        spearman = float(np.corrcoef(rc, rt)[0, 1]) if len(timed) > 2 else None
        same = [x[0] for x in timed if x[2] == pick[0]]
        rows.append({"pattern": name, "count": count, "configs": len(timed),
                     "measured_whole": sum(1 for x in timed if x[4]),
                     "best_s": best, "worst_s": max(times), "pick_s": pick_t,
                     "pick_vs_best": pick_t / best, "worst_vs_best": max(times) / best,
                     "spearman_cost_vs_time": spearman,
                     "sets_for_pick_schedule": len(same),
                     "pick_set_vs_best_set_same_schedule": pick_t / min(same) if same else None,
                     "mean_set_vs_best_set_same_schedule": float(np.mean(same)) / min(same) if same else None})
        print(json.dumps(rows[-1], default=str), file=sys.stderr, flush=True)
    return {"metric": "performance-model accuracy", "graph": graph_name, "iep": iep,
            "timing": f"whole counts below {limit_s} s, else projections (busy warp cycles) from the same "
                      "1024 x 64-task sample",
            "rows": rows}


def plan_bench(repeats=3):
    """Host planning time per named pattern (Section IV-A to IV-C: the
    automorphisms, Algorithm 1's restriction sets, the efficient schedules
    and the top-3 ranking by the performance model with default graph
    statistics), best of `repeats` on a fresh pattern handle each time; the
    counterpart of the paper's preprocessing times (Table III)."""
    from paper_2009_10955_gb300 import native
    from synth.patterns import NAMED_PATTERNS
    N = native()
    rows = {}
    for name in NAMED_PATTERNS:
        adj = named_pattern(name)
        best = None
        for _ in range(repeats):
            t = time.perf_counter()
            p = N.gp_pattern_create(adj)
            sc = N.gp_schedule(p, None, top_k=3)
            dt = time.perf_counter() - t
            best = dt if best is None else min(best, dt)
        rows[name] = {"k": int(adj.shape[0]), "aut": p.aut_count(), "restriction_sets": len(p.restriction_sets()),
                      "schedules": len(p.schedules()[0]), "plans": len(sc), "plan_ms": best * 1000.0}
    return {"metric": "host planning time (ms)", "unit": "ms", "cores": 1,
            "host": os.uname().machine, "timing": f"best of {repeats}, fresh pattern handle each time",
            "patterns": rows}


def reference_arm(a):
    """The oracle on the host cores, each step a bounded random root sample."""
    wl = WORKLOADS[a.workload]
    pats = a.patterns.split(",") if a.patterns else wl["patterns"]
    n, src, dst = workload_edges(wl["graph"])
    import oracle
    ref = oracle.build_csr(n, src, dst)
    deg = np.diff(ref.row_ptr)
    config = workload_config(a.workload, wl["graph"], n, int(ref.row_ptr[-1]) // 2,
                             int(deg.max()) if n else 0, pats)
    del ref, deg
    per_step = max(2.0, 150.0 / max(1, a.steps + a.warmup))
    vals = []
    cb = None
    for i in range(a.warmup + a.steps):
        cb = cpu_baseline(n, src, dst, pats, per_step)
        if i >= a.warmup:
            vals.append(cb["value"])
    v = statistics.mean(vals)
    cb["value"] = v
    return {"metric": "pattern-count time (s)", "value": v, "unit": "s", "n_gpus": a.gpus, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": v * 1000.0, "higher_is_better": False, "impl": "reference",
            "scaling": "strong", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": config,
            "method": {"step": "one bounded, degree-stratified root sample of each pattern",
                       "parallelism": "host cores (the oracle runs on the CPU; rank 0 alone)"},
            "devices": "host cores only (the oracle runs on the CPU; rank 0 alone)",
            "cpu_baseline": cb,
            "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    a = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if a.impl == "reference":
        if rank == 0:
            print(json.dumps(reference_arm(a)), flush=True)
        return
    if a.mode == "plan":
        if rank == 0:
            print(json.dumps(plan_bench()), flush=True)
        return
    import torch
    if a.mode == "model":
        if rank == 0:
            from paper_2009_10955_gb300 import native
            out = model_bench(native(), torch.cuda.current_stream(), a.model_graph, a.model_patterns.split(","),
                              iep=not a.no_iep)
            print(json.dumps(out, default=str), flush=True)
        return
    if a.mode == "directed":
        if rank == 0:
            from paper_2009_10955_gb300 import native
            print(json.dumps(directed_bench(native(), torch.cuda.current_stream())), flush=True)
        return
    if a.mode == "iep":
        if rank == 0:
            from paper_2009_10955_gb300 import native
            cases = [tuple(x.split("/")) for x in a.iep_cases.split(",")]
            print(json.dumps(iep_bench(native(), torch.cuda.current_stream(), cases), default=str), flush=True)
        return
    if a.mode == "case":
        # graph (degree order), its triangle count for the performance model
        # (the first count-kernel launch), then one count of each pattern
        if rank == 0:
            from paper_2009_10955_gb300 import native
            N = native()
            n, src, dst = workload_edges(a.graph)
            g = N.gp_graph_create_edges(src, dst, n, N.GP_DEGREE_ORDER)
            g.stats()
            nnz = g.device_csr()[2]
            lo_f, hi_f = (float(x) for x in a.case_range.split(","))
            tb, te = int(nnz * lo_f), int(nnz * hi_f)
            for pn in (a.patterns or "k4").split(","):
                if a.model_plan:
                    sc = N.gp_schedule(N.gp_pattern_create(named_pattern(pn)), g)
                    if not a.no_iep:
                        sc.set_iep(True)
                else:
                    from paper_2009_10955_gb300 import autotune
                    cache = os.path.join(ROOT, "paper_2009_10955_gb300", "_build", "tune_cache.json")
                    sc, _ = autotune.choose_plan(g, named_pattern(pn), top_k=3, iep=not a.no_iep, cache_path=cache)
                print(pn, sc.get(0)[:2], sc.iep(0),
                      N.gp_count_raw(g, sc, 0, task_begin=tb, task_end=te if te < nnz else 0), flush=True)
            torch.cuda.synchronize()
        return
    if a.mode == "serve":
        if rank == 0:
            from paper_2009_10955_gb300 import native
            N = native()
            out = serve_bench(N, torch.cuda.current_stream(), [int(x) for x in a.serve_scales.split(",")],
                              [float(x) for x in a.serve_rates.split(",")], a.serve_requests,
                              a.serve_deadline, a.serve_slice_ms,
                              mem_budget=int(a.serve_mem_gb * (1 << 30)) if a.serve_mem_gb > 0 else None)
            print(json.dumps(out), flush=True)
        return
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        dist.init_process_group("nccl")
    out, (n, src, dst, pats) = gpu_arm(a, rank, world)
    if rank == 0:
        if world == 1 and not a.no_cpu_baseline:
            phase("cpu baseline")
            out["cpu_baseline"] = cpu_baseline(n, src, dst, pats, a.cpu_seconds)
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
