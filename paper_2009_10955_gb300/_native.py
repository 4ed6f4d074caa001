"""ctypes binding of libgraphpi_gb300.so: the C ABI of include/graphpi.h under
the same names, plus small handle classes that call ``*_destroy``.

This module only marshals arguments. Every step of the counting path runs in
the library's CUDA kernels; when the library is missing the import raises,
there is no fallback.
"""

import ctypes
import os

import numpy as np

from . import build as _build

GP_OK = 0
GP_PARTIAL = 1
GP_ERR_ARG = -1
GP_ERR_PATTERN = -2
GP_ERR_NOMEM = -3
GP_ERR_CUDA = -4
GP_ERR_OVERFLOW = -5
GP_ERR_TIMEOUT = -6
GP_ERR_SCRATCH = -7
GP_ERR_INTERNAL = -8

GP_DEVICE_PTRS = 1
GP_DEGREE_ORDER = 2
GP_ASSUME_CLEAN = 4
GP_COUNT_STATS = 1
GP_COUNT_NO_CORE = 2
GP_COUNT_WARP_BITMAP = 4
GP_COUNT_LANE_BITMAP = 8

# Every function the header declares, with its ctypes signature.
P = ctypes.c_void_p
i32, i64, u32, f64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32, ctypes.c_double
SIGNATURES = {
    "gp_graph_create_edges": (i32, [P, P, i64, i32, u32, P, P]),
    "gp_graph_create_csr": (i32, [P, P, i32, u32, P, P]),
    "gp_graph_stats": (i32, [P, P, P, P, P, P]),
    "gp_graph_copy_csr": (i32, [P, P, P, P]),
    "gp_graph_device_csr": (i32, [P, P, P, P]),
    "gp_graph_destroy": (None, [P]),
    "gp_pattern_create": (i32, [P, i32, P]),
    "gp_pattern_aut_count": (i32, [P, P]),
    "gp_pattern_create_labeled": (i32, [P, P, i32, P]),
    "gp_graph_set_labels": (i32, [P, P, P]),
    "gp_pattern_restriction_sets": (i32, [P, i32, P, i32, P, P]),
    "gp_pattern_schedules": (i32, [P, P, P, i32, P]),
    "gp_pattern_destroy": (None, [P]),
    "gp_schedule": (i32, [P, P, i32, P, P]),
    "gp_schedule_explicit": (i32, [P, P, P, i32, P]),
    "gp_schedule_size": (i32, [P, P]),
    "gp_schedule_set_iep": (i32, [P, i32, P]),
    "gp_schedule_iep": (i32, [P, i32, P, P]),
    "gp_schedule_get": (i32, [P, i32, P, P, P, P]),
    "gp_config_cost": (i32, [P, P, P, i32, f64, f64, f64, P]),
    "gp_schedule_destroy": (None, [P]),
    "gp_count": (i32, [P, P, i32, P, P, P]),
    "gp_count_batch": (i32, [P, P, P, i32, P, P, P]),
    "gp_count_batch_ranges": (i32, [P, P, P, P, P, i32, P, P, P, P]),
    "gp_count_scratch_bytes": (i32, [P, P, i32, P, P]),
    "gp_count_noalloc": (i32, [P, P, i32, P, P]),
    "gp_list": (i32, [P, P, i32, i64, i64, P, i64, P, P, P]),
    "gp_dgraph_create": (i32, [P, P, i64, i32, u32, P, P]),
    "gp_dgraph_stats": (i32, [P, P, P]),
    "gp_dgraph_copy": (i32, [P, P, P, P, P]),
    "gp_dgraph_destroy": (None, [P]),
    "gp_dpattern_create": (i32, [P, i32, P]),
    "gp_dpattern_aut_count": (i32, [P, P]),
    "gp_dpattern_destroy": (None, [P]),
    "gp_dcount": (i32, [P, P, P, P, i32, P, P]),
    "gp_status_str": (ctypes.c_char_p, [i32]),
    "gp_last_error": (ctypes.c_char_p, []),
    "gp_take_launch_count": (i64, []),
}


class gp_count_opts(ctypes.Structure):
    _fields_ = [
        ("struct_size", ctypes.c_int32),
        ("warps_per_block", ctypes.c_int32),
        ("blocks_per_sm", ctypes.c_int32),
        ("chunk", ctypes.c_int32),
        ("split", ctypes.c_int32),
        ("flags", ctypes.c_int32),
        ("task_begin", ctypes.c_int64),
        ("task_end", ctypes.c_int64),
        ("budget_cycles", ctypes.c_int64),
        ("resume_cursor", ctypes.POINTER(ctypes.c_int64)),
        ("kernel_ms", ctypes.POINTER(ctypes.c_float)),
        ("algo_bytes", ctypes.POINTER(ctypes.c_uint64)),
        ("lane_work", ctypes.c_int32),
        ("reserved1", ctypes.c_int32),
        ("task_cycles", ctypes.c_int64),
        ("raw_total", ctypes.POINTER(ctypes.c_uint64)),
        ("algo_ops", ctypes.POINTER(ctypes.c_uint64)),
        ("busy_cycles", ctypes.POINTER(ctypes.c_uint64)),
    ]


def make_opts(**kw):
    o = gp_count_opts()
    o.struct_size = ctypes.sizeof(gp_count_opts)
    for k, v in kw.items():
        setattr(o, k, v)
    return o


_lib = None


def load(build_if_missing=True):
    """Load the library (building it first when it is missing or stale)."""
    global _lib
    if _lib is None:
        if build_if_missing and not _build.up_to_date():
            _build.build()
        if not os.path.exists(_build.LIB):
            raise ImportError(f"libgraphpi_gb300.so is not built ({_build.LIB})")
        lib = ctypes.CDLL(_build.LIB)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
    return _lib


def lib():
    return load()


class GraphPiError(RuntimeError):
    def __init__(self, status, where):
        L = lib()
        msg = L.gp_last_error().decode(errors="replace")
        super().__init__(f"{where}: {L.gp_status_str(status).decode()} ({status}): {msg}")
        self.status = status


def check(status, where):
    if status < 0:
        raise GraphPiError(status, where)
    return status


def _ptr(a):
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data_as(ctypes.c_void_p)
    if hasattr(a, "data_ptr"):          # torch tensor
        return ctypes.c_void_p(a.data_ptr())
    return ctypes.c_void_p(int(a))


def _stream(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


# ------------------------------------------------------------ same-name calls

def gp_graph_create_edges(src, dst, n, flags=0, stream=None):
    """Returns a Graph. src/dst: int32 numpy arrays (host) or, with
    GP_DEVICE_PTRS, int32 device tensors."""
    if isinstance(src, np.ndarray):
        src = np.ascontiguousarray(src, dtype=np.int32)
        dst = np.ascontiguousarray(dst, dtype=np.int32)
    m = int(src.shape[0]) if hasattr(src, "shape") else len(src)
    h = ctypes.c_void_p()
    check(lib().gp_graph_create_edges(_ptr(src), _ptr(dst), m, int(n), flags, _stream(stream),
                                      ctypes.byref(h)), "gp_graph_create_edges")
    return Graph(h)


def gp_graph_create_csr(row_ptr, col, n, flags=0, stream=None):
    if isinstance(row_ptr, np.ndarray):
        row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
        col = np.ascontiguousarray(col, dtype=np.int32)
    h = ctypes.c_void_p()
    check(lib().gp_graph_create_csr(_ptr(row_ptr), _ptr(col), int(n), flags, _stream(stream),
                                    ctypes.byref(h)), "gp_graph_create_csr")
    return Graph(h)


def gp_pattern_create(adj):
    adj = np.ascontiguousarray(adj, dtype=np.uint8)
    if adj.ndim != 2 or adj.shape[0] != adj.shape[1]:
        raise ValueError("adjacency must be k x k")
    h = ctypes.c_void_p()
    check(lib().gp_pattern_create(_ptr(adj), adj.shape[0], ctypes.byref(h)), "gp_pattern_create")
    return Pattern(h, adj.shape[0])


def gp_pattern_create_labeled(adj, labels):
    adj = np.ascontiguousarray(adj, dtype=np.uint8)
    lab = np.ascontiguousarray(labels, dtype=np.int32)
    h = ctypes.c_void_p()
    check(lib().gp_pattern_create_labeled(_ptr(adj), _ptr(lab), adj.shape[0], ctypes.byref(h)),
          "gp_pattern_create_labeled")
    return Pattern(h, adj.shape[0])


def gp_graph_set_labels(graph, labels, stream=None):
    lab = np.ascontiguousarray(labels, dtype=np.int32)
    check(lib().gp_graph_set_labels(graph.h, _ptr(lab), _stream(stream)), "gp_graph_set_labels")


def gp_schedule(pattern, graph=None, top_k=1, stream=None):
    h = ctypes.c_void_p()
    check(lib().gp_schedule(pattern.h, graph.h if graph is not None else None, top_k, _stream(stream),
                            ctypes.byref(h)), "gp_schedule")
    return Schedules(h, pattern.k)


def gp_schedule_explicit(pattern, order, restrictions):
    order = np.ascontiguousarray(order, dtype=np.int32)
    res = np.ascontiguousarray(np.array(restrictions, dtype=np.int32).reshape(-1, 2))
    h = ctypes.c_void_p()
    check(lib().gp_schedule_explicit(pattern.h, _ptr(order), _ptr(res) if res.size else None,
                                     res.shape[0], ctypes.byref(h)), "gp_schedule_explicit")
    return Schedules(h, pattern.k)


def gp_count(graph, schedules, idx=0, opts=None, stream=None):
    """Returns (status, count); status is GP_OK or GP_PARTIAL."""
    out = ctypes.c_uint64()
    st = check(lib().gp_count(graph.h, schedules.h, idx, ctypes.byref(opts) if opts is not None else None,
                              _stream(stream), ctypes.byref(out)), "gp_count")
    return st, out.value


def gp_count_raw(graph, schedules, idx=0, opts=None, stream=None, **kw):
    """Returns (status, raw): the undivided 128-bit total of the processed
    tasks as a Python int (the count for plain plans; count x divisor for
    inclusion-exclusion plans). Extra keywords go to make_opts."""
    raw = (ctypes.c_uint64 * 2)()
    o = opts if opts is not None else make_opts(**kw)
    o.raw_total = ctypes.cast(raw, ctypes.POINTER(ctypes.c_uint64))
    out = ctypes.c_uint64()
    st = check(lib().gp_count(graph.h, schedules.h, idx, ctypes.byref(o), _stream(stream), ctypes.byref(out)),
               "gp_count")
    return st, int(raw[0]) | (int(raw[1]) << 64)


def gp_count_batch(graphs, schedules, idx=None, opts=None, stream=None, raw=None):
    """Counts of the jobs (uint64 array). With raw (a uint64 numpy array of
    2 x len(graphs)), the undivided 128-bit totals (low, high) are written
    there, and counts beyond 64 bits come back as 0 instead of failing."""
    n = len(graphs)
    G = (ctypes.c_void_p * n)(*[g.h.value for g in graphs])
    S = (ctypes.c_void_p * n)(*[s.h.value for s in schedules])
    I = np.ascontiguousarray(idx if idx is not None else np.zeros(n), dtype=np.int32)
    out = np.zeros(n, dtype=np.uint64)
    if raw is not None:
        if opts is None:
            opts = make_opts()
        opts.raw_total = raw.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))
    check(lib().gp_count_batch(G, S, _ptr(I), n, ctypes.byref(opts) if opts is not None else None,
                               _stream(stream), _ptr(out)), "gp_count_batch")
    return out


def gp_count_batch_ranges(graphs, schedules, idx, task_begin, task_end, opts=None, stream=None, raw=None):
    """Returns (status, counts, next_task) for one time slice. With raw (a
    uint64 numpy array of 2 x len(graphs)), the undivided 128-bit totals
    (low, high) are written there; inclusion-exclusion jobs need it."""
    n = len(graphs)
    G = (ctypes.c_void_p * n)(*[g.h.value for g in graphs])
    S = (ctypes.c_void_p * n)(*[s.h.value for s in schedules])
    I = np.ascontiguousarray(idx, dtype=np.int32)
    B = np.ascontiguousarray(task_begin, dtype=np.int64)
    E = np.ascontiguousarray(task_end, dtype=np.int64)
    out = np.zeros(n, dtype=np.uint64)
    nxt = np.zeros(n, dtype=np.int64)
    if raw is not None:
        if opts is None:
            opts = make_opts()
        opts.raw_total = raw.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))
    st = check(lib().gp_count_batch_ranges(G, S, _ptr(I), _ptr(B), _ptr(E), n,
                                           ctypes.byref(opts) if opts is not None else None,
                                           _stream(stream), _ptr(out), _ptr(nxt)), "gp_count_batch_ranges")
    return st, out, nxt


def gp_count_scratch_bytes(graph, schedules, idx=0, opts=None):
    out = ctypes.c_uint64()
    check(lib().gp_count_scratch_bytes(graph.h, schedules.h, idx, ctypes.byref(opts) if opts is not None else None,
                                       ctypes.byref(out)), "gp_count_scratch_bytes")
    return out.value


def gp_config_cost(pattern, order, restrictions, n_vertices, n_edges, tri_cnt):
    order = np.ascontiguousarray(order, dtype=np.int32)
    res = np.ascontiguousarray(np.array(restrictions, dtype=np.int32).reshape(-1, 2))
    out = ctypes.c_double()
    check(lib().gp_config_cost(pattern.h, _ptr(order), _ptr(res) if res.size else None, res.shape[0],
                               float(n_vertices), float(n_edges), float(tri_cnt), ctypes.byref(out)),
          "gp_config_cost")
    return out.value


def gp_count_noalloc(graph, schedules, idx=0, stream=None):
    """Count with the library's fixed device scratch (no allocation)."""
    out = ctypes.c_uint64()
    check(lib().gp_count_noalloc(graph.h, schedules.h, idx, _stream(stream), ctypes.byref(out)),
          "gp_count_noalloc")
    return out.value


def gp_list(graph, schedules, idx, task_begin, task_end, out, capacity, stream=None):
    """List embeddings into the device buffer `out` (capacity x k int32, e.g.
    a torch tensor). Returns (status, n_written, next_task)."""
    nw, nt = ctypes.c_int64(), ctypes.c_int64()
    st = check(lib().gp_list(graph.h, schedules.h, idx, int(task_begin), int(task_end), _ptr(out), int(capacity),
                             _stream(stream), ctypes.byref(nw), ctypes.byref(nt)), "gp_list")
    return st, nw.value, nt.value


def gp_dgraph_create(src, dst, n, flags=0, stream=None):
    """Directed graph of arcs src[i] -> dst[i] (int32 numpy arrays, or device
    tensors with GP_DEVICE_PTRS). Returns a DGraph."""
    if isinstance(src, np.ndarray):
        src = np.ascontiguousarray(src, dtype=np.int32)
        dst = np.ascontiguousarray(dst, dtype=np.int32)
    m = int(src.shape[0]) if hasattr(src, "shape") else len(src)
    h = ctypes.c_void_p()
    check(lib().gp_dgraph_create(_ptr(src), _ptr(dst), m, int(n), flags, _stream(stream), ctypes.byref(h)),
          "gp_dgraph_create")
    return DGraph(h)


def gp_dpattern_create(adj):
    """Directed pattern: adj[a, b] = 1 for an arc a -> b."""
    adj = np.ascontiguousarray(adj, dtype=np.uint8)
    if adj.ndim != 2 or adj.shape[0] != adj.shape[1]:
        raise ValueError("adjacency must be k x k")
    h = ctypes.c_void_p()
    check(lib().gp_dpattern_create(_ptr(adj), adj.shape[0], ctypes.byref(h)), "gp_dpattern_create")
    return DPattern(h, adj.shape[0])


def gp_dcount(graph, pattern, order=None, restrictions=None, stream=None):
    """Count; with order=None the planner chooses the configuration; with an
    order, restrictions=[] counts without restrictions (dividing by |Aut|)."""
    out = ctypes.c_uint64()
    if order is None:
        check(lib().gp_dcount(graph.h, pattern.h, None, None, 0, _stream(stream), ctypes.byref(out)), "gp_dcount")
        return out.value
    o = np.ascontiguousarray(order, dtype=np.int32)
    res = np.ascontiguousarray(np.array(restrictions or [], dtype=np.int32).reshape(-1, 2))
    check(lib().gp_dcount(graph.h, pattern.h, _ptr(o), _ptr(res) if res.size else None, res.shape[0],
                          _stream(stream), ctypes.byref(out)), "gp_dcount")
    return out.value


def gp_take_launch_count():
    return int(lib().gp_take_launch_count())


# ------------------------------------------------------------------- handles

class Graph:
    def __init__(self, h):
        self.h = h

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.gp_graph_destroy(self.h)
            self.h = None

    def stats(self, with_triangles=True, stream=None):
        n, m, md, t = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int32(), ctypes.c_uint64()
        check(lib().gp_graph_stats(self.h, ctypes.byref(n), ctypes.byref(m), ctypes.byref(md),
                                   ctypes.byref(t) if with_triangles else None, _stream(stream)),
              "gp_graph_stats")
        return {"n": n.value, "m": m.value, "max_deg": md.value, "tri_cnt": t.value if with_triangles else None}

    def csr(self):
        s = self.stats(with_triangles=False)
        row_ptr = np.zeros(s["n"] + 1, dtype=np.int64)
        col = np.zeros(max(1, 2 * s["m"]), dtype=np.int32)
        perm = np.zeros(max(1, s["n"]), dtype=np.int32)
        check(lib().gp_graph_copy_csr(self.h, _ptr(row_ptr), _ptr(col), _ptr(perm)), "gp_graph_copy_csr")
        return row_ptr, col[: 2 * s["m"]], perm[: s["n"]]

    def device_csr(self):
        rp, cl, nnz = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_int64()
        check(lib().gp_graph_device_csr(self.h, ctypes.byref(rp), ctypes.byref(cl), ctypes.byref(nnz)),
              "gp_graph_device_csr")
        return rp.value, cl.value, nnz.value


class Pattern:
    def __init__(self, h, k):
        self.h = h
        self.k = k

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.gp_pattern_destroy(self.h)
            self.h = None

    def aut_count(self):
        out = ctypes.c_uint64()
        check(lib().gp_pattern_aut_count(self.h, ctypes.byref(out)), "gp_pattern_aut_count")
        return out.value

    def restriction_sets(self, cap=0):
        cnt = ctypes.c_int32()
        check(lib().gp_pattern_restriction_sets(self.h, cap, ctypes.byref(cnt), 0, None, None),
              "gp_pattern_restriction_sets")
        out = []
        pairs = np.zeros(64, dtype=np.int32)
        npairs = ctypes.c_int32()
        for i in range(cnt.value):
            check(lib().gp_pattern_restriction_sets(self.h, cap, ctypes.byref(cnt), i, _ptr(pairs),
                                                    ctypes.byref(npairs)), "gp_pattern_restriction_sets")
            out.append(tuple((int(pairs[2 * r]), int(pairs[2 * r + 1])) for r in range(npairs.value)))
        return out

    def schedules(self):
        cnt, kp = ctypes.c_int32(), ctypes.c_int32()
        check(lib().gp_pattern_schedules(self.h, ctypes.byref(cnt), ctypes.byref(kp), 0, None),
              "gp_pattern_schedules")
        order = np.zeros(8, dtype=np.int32)
        out = []
        for i in range(cnt.value):
            check(lib().gp_pattern_schedules(self.h, ctypes.byref(cnt), ctypes.byref(kp), i, _ptr(order)),
                  "gp_pattern_schedules")
            out.append(tuple(int(x) for x in order[: self.k]))
        return out, kp.value


class Schedules:
    def __init__(self, h, k):
        self.h = h
        self.k = k

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.gp_schedule_destroy(self.h)
            self.h = None

    def set_iep(self, enable=True):
        n = ctypes.c_int32()
        check(lib().gp_schedule_set_iep(self.h, 1 if enable else 0, ctypes.byref(n)), "gp_schedule_set_iep")
        return n.value

    def iep(self, idx=0):
        """(kk, divisor) of plan idx: kk innermost loops replaced by
        inclusion-exclusion (0: none), undivided totals divided by divisor."""
        kk, div = ctypes.c_int32(), ctypes.c_uint32()
        check(lib().gp_schedule_iep(self.h, idx, ctypes.byref(kk), ctypes.byref(div)), "gp_schedule_iep")
        return kk.value, div.value

    def __len__(self):
        c = ctypes.c_int32()
        check(lib().gp_schedule_size(self.h, ctypes.byref(c)), "gp_schedule_size")
        return c.value

    def get(self, idx):
        order = np.zeros(8, dtype=np.int32)
        res = np.zeros(64, dtype=np.int32)
        nres = ctypes.c_int32()
        cost = ctypes.c_double()
        check(lib().gp_schedule_get(self.h, idx, _ptr(order), _ptr(res), ctypes.byref(nres), ctypes.byref(cost)),
              "gp_schedule_get")
        return (tuple(int(x) for x in order[: self.k]),
                tuple((int(res[2 * r]), int(res[2 * r + 1])) for r in range(nres.value)),
                cost.value)


class DGraph:
    def __init__(self, h):
        self.h = h

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.gp_dgraph_destroy(self.h)
            self.h = None

    def stats(self):
        n, a = ctypes.c_int64(), ctypes.c_int64()
        check(lib().gp_dgraph_stats(self.h, ctypes.byref(n), ctypes.byref(a)), "gp_dgraph_stats")
        return {"n": n.value, "narcs": a.value}

    def lists(self):
        s = self.stats()
        op, ip = np.zeros(s["n"] + 1, np.int64), np.zeros(s["n"] + 1, np.int64)
        oc, ic = np.zeros(max(1, s["narcs"]), np.int32), np.zeros(max(1, s["narcs"]), np.int32)
        check(lib().gp_dgraph_copy(self.h, _ptr(op), _ptr(oc), _ptr(ip), _ptr(ic)), "gp_dgraph_copy")
        return op, oc[: s["narcs"]], ip, ic[: s["narcs"]]


class DPattern:
    def __init__(self, h, k):
        self.h = h
        self.k = k

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.gp_dpattern_destroy(self.h)
            self.h = None

    def aut_count(self):
        out = ctypes.c_uint64()
        check(lib().gp_dpattern_aut_count(self.h, ctypes.byref(out)), "gp_dpattern_aut_count")
        return out.value

