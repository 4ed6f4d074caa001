"""Oracle for the GraphPi pattern-count path.

TEST INFRASTRUCTURE ONLY. Only the tests, the smoke check and the benchmark's
CPU-baseline leg may import this package. The counting library never imports
it, and the two share no code: this package reads its inputs from the seeded
generators in ``synth`` (which hold none of the method's arithmetic) and
builds its own CSR, automorphism group, restriction sets, schedules and cost
model from the paper's definitions.

* ``oracle.c`` (plain C11 + pthreads): CSR build, |Aut(P)|, injective map
  enumeration, restricted enumeration, listing, triangles (Sections II-A,
  II-B, IV-E); vertex-labelled counts; directed patterns on graphs with
  out- and in-lists (the paper names directed patterns without defining
  them; an embedding sends every pattern arc to a graph arc).
* ``planner_ref.py`` (plain Python): automorphisms, Algorithm 1 with
  ``no_conflict`` and ``validate``, the 2-phase schedule filter and the
  performance model (Sections IV-A to IV-C), Algorithm 2 and the
  inclusion-exclusion count of distinct tuples (Section IV-D).
* ``iep_total`` (here): a whole count with the innermost loops replaced by
  that inclusion-exclusion count (Section IV-D), on small graphs.

Parity status: every function here is pinned by ``tests/test_oracle_pins.py``,
``tests/test_oracle_pins_directed.py``, ``tests/test_golden_paper.py``,
``tests/test_cost_pins.py``, ``tests/test_iep_divisor.py`` and
``tests/test_iep_partitions.py`` (closed forms, brute force over vertex
tuples, values the paper prints); the mutation tests show that the pins
catch planted mistakes.
"""

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None


def build(force=False):
    """Compile ``oracle.c`` with gcc into ``oracle/_build/liboracle.so``."""
    src = os.path.join(_HERE, "oracle.c")
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= max(
            os.path.getmtime(src), os.path.getmtime(os.path.join(_HERE, "oracle.h"))):
        return _SO
    os.makedirs(os.path.dirname(_SO), exist_ok=True)
    tmp = _SO + f".{os.getpid()}.tmp"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-Wall", "-fPIC", "-shared", "-pthread",
                           src, "-o", tmp])
    os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is None:
        _lib = configure(ctypes.CDLL(build()))
    return _lib


def configure(lib):
    """Declare the C signatures on a loaded copy of ``oracle.c``'s library."""
    P = ctypes.c_void_p
    i32, i64 = ctypes.c_int32, ctypes.c_int64
    lib.oracle_build_csr.argtypes = [i32, i64, P, P, P, P, P]
    lib.oracle_aut_count.argtypes = [i32, P, P]
    lib.oracle_count_maps.argtypes = [i32, P, i32, P, P, i32, i32, i32, i32, P, P]
    lib.oracle_count_restricted.argtypes = [i32, P, P, i32, P, i32, P, P, i32, i32, i32, P, P]
    lib.oracle_count_restricted_entries.argtypes = [i32, P, P, i32, P, i32, P, P, i64, i64, i32, P, P]
    lib.oracle_count_restricted_entries.restype = ctypes.c_int
    lib.oracle_triangles.argtypes = [i32, P, P, i32, P]
    lib.oracle_list_restricted.argtypes = [i32, P, P, i32, P, i32, P, P, i32, i32, P, i64, P]
    lib.oracle_list_restricted.restype = ctypes.c_int
    lib.oracle_aut_count_labeled.argtypes = [i32, P, P, P]
    lib.oracle_aut_count_labeled.restype = ctypes.c_int
    lib.oracle_count_labeled.argtypes = [i32, P, P, i32, P, P, P, i32, P]
    lib.oracle_count_labeled.restype = ctypes.c_int
    lib.oracle_build_dcsr.argtypes = [i32, i64, P, P, P, P, P, P, P]
    lib.oracle_aut_count_directed.argtypes = [i32, P, P]
    lib.oracle_count_directed.argtypes = [i32, P, P, i32, P, i32, P, P, P, P, i32, i32, i32, P, P]
    for f in (lib.oracle_build_csr, lib.oracle_aut_count, lib.oracle_count_maps,
              lib.oracle_count_restricted, lib.oracle_triangles, lib.oracle_build_dcsr,
              lib.oracle_aut_count_directed, lib.oracle_count_directed):
        f.restype = ctypes.c_int
    return lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def default_threads():
    return os.cpu_count() or 1


class Csr:
    """Undirected simple graph in CSR form (int64 row_ptr, int32 col)."""

    def __init__(self, n, row_ptr, col):
        self.n = int(n)
        self.row_ptr = row_ptr
        self.col = col

    @property
    def nnz(self):
        return int(self.row_ptr[-1])


def build_csr(n, src, dst):
    src = np.ascontiguousarray(src, dtype=np.int32)
    dst = np.ascontiguousarray(dst, dtype=np.int32)
    m = len(src)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    col = np.zeros(max(1, 2 * m), dtype=np.int32)
    nnz = np.zeros(1, dtype=np.int64)
    rc = _load().oracle_build_csr(n, m, _p(src), _p(dst), _p(row_ptr), _p(col), _p(nnz))
    if rc:
        raise ValueError(f"oracle_build_csr failed ({rc})")
    return Csr(n, row_ptr, col[: int(nnz[0])].copy())


def _adj(adj):
    adj = np.ascontiguousarray(adj, dtype=np.uint8)
    if adj.ndim != 2 or adj.shape[0] != adj.shape[1]:
        raise ValueError("adjacency must be k x k")
    return adj


def aut_count(adj):
    adj = _adj(adj)
    out = np.zeros(1, dtype=np.uint64)
    rc = _load().oracle_aut_count(adj.shape[0], _p(adj), _p(out))
    if rc:
        raise ValueError(f"oracle_aut_count failed ({rc})")
    return int(out[0])


def count_maps(adj, g, root_begin=0, root_end=None, root_stride=1, threads=None):
    """Injective edge-preserving maps (as a Python int) with the image of
    pattern vertex 0 among the selected roots."""
    adj = _adj(adj)
    hi = np.zeros(1, dtype=np.uint64)
    lo = np.zeros(1, dtype=np.uint64)
    rc = _load().oracle_count_maps(adj.shape[0], _p(adj), g.n, _p(g.row_ptr), _p(g.col),
                                   root_begin, g.n if root_end is None else root_end,
                                   root_stride, threads or default_threads(), _p(hi), _p(lo))
    if rc:
        raise ValueError(f"oracle_count_maps failed ({rc})")
    return (int(hi[0]) << 64) | int(lo[0])


def count(adj, g, threads=None):
    """count(P, G) = maps / |Aut(P)|, as a Python int (may exceed 64 bits)."""
    maps = count_maps(adj, g, threads=threads)
    aut = aut_count(adj)
    if maps % aut:
        raise AssertionError("map count is not a multiple of |Aut(P)|")
    return maps // aut


def count_restricted(adj, order, restrictions, g, threads=None, root_begin=0, root_end=None):
    """Maps found in matching order ``order`` that obey every restriction
    ``(a, b)``: id(a) > id(b), with the first searched vertex's image in
    ``[root_begin, root_end)``."""
    adj = _adj(adj)
    k = adj.shape[0]
    order = np.ascontiguousarray(order, dtype=np.int32)
    res = np.ascontiguousarray(np.array(restrictions, dtype=np.int32).reshape(-1, 2))
    if res.size == 0:
        res = np.zeros((1, 2), dtype=np.int32)
        nres = 0
    else:
        nres = res.shape[0]
    hi = np.zeros(1, dtype=np.uint64)
    lo = np.zeros(1, dtype=np.uint64)
    rc = _load().oracle_count_restricted(k, _p(adj), _p(order), nres, _p(res), g.n,
                                         _p(g.row_ptr), _p(g.col), root_begin,
                                         g.n if root_end is None else root_end,
                                         threads or default_threads(), _p(hi), _p(lo))
    if rc:
        raise ValueError(f"oracle_count_restricted failed ({rc})")
    return (int(hi[0]) << 64) | int(lo[0])


def count_restricted_entries(adj, order, restrictions, g, entry_begin, entry_end, threads=None):
    """count_restricted over the maps whose first two searched vertices are
    a CSR entry (row, column) in ``[entry_begin, entry_end)``."""
    adj = _adj(adj)
    k = adj.shape[0]
    order = np.ascontiguousarray(order, dtype=np.int32)
    res = np.ascontiguousarray(np.array(restrictions, dtype=np.int32).reshape(-1, 2))
    nres = res.shape[0] if res.size else 0
    if res.size == 0:
        res = np.zeros((1, 2), dtype=np.int32)
    hi = np.zeros(1, dtype=np.uint64)
    lo = np.zeros(1, dtype=np.uint64)
    rc = _load().oracle_count_restricted_entries(k, _p(adj), _p(order), nres, _p(res), g.n,
                                                 _p(g.row_ptr), _p(g.col), int(entry_begin), int(entry_end),
                                                 threads or default_threads(), _p(hi), _p(lo))
    if rc:
        raise ValueError(f"oracle_count_restricted_entries failed ({rc})")
    return (int(hi[0]) << 64) | int(lo[0])


def list_restricted(adj, order, restrictions, g, root_begin=0, root_end=None, cap=1 << 22):
    """Embeddings (k-tuples, entry a = image of pattern vertex a) found in
    matching order `order` under the restrictions; returns (array, total)."""
    adj = _adj(adj)
    k = adj.shape[0]
    order = np.ascontiguousarray(order, dtype=np.int32)
    res = np.ascontiguousarray(np.array(restrictions, dtype=np.int32).reshape(-1, 2))
    nres = res.shape[0]
    if nres == 0:
        res = np.zeros((1, 2), dtype=np.int32)
    out = np.zeros((max(1, cap), k), dtype=np.int32)
    n_out = np.zeros(1, dtype=np.int64)
    rc = _load().oracle_list_restricted(k, _p(adj), _p(order), nres, _p(res), g.n, _p(g.row_ptr),
                                        _p(g.col), root_begin, g.n if root_end is None else root_end,
                                        _p(out), cap, _p(n_out))
    if rc:
        raise ValueError(f"oracle_list_restricted failed ({rc})")
    total = int(n_out[0])
    return out[: min(total, cap)].copy(), total


def aut_count_labeled(adj, plabels):
    adj = _adj(adj)
    pl = np.ascontiguousarray(plabels, dtype=np.int32)
    out = np.zeros(1, dtype=np.uint64)
    rc = _load().oracle_aut_count_labeled(adj.shape[0], _p(adj), _p(pl), _p(out))
    if rc:
        raise ValueError(f"oracle_aut_count_labeled failed ({rc})")
    return int(out[0])


def count_labeled(adj, plabels, g, glabels, threads=None):
    """Embeddings of a vertex-labelled pattern in a vertex-labelled graph."""
    adj = _adj(adj)
    pl = np.ascontiguousarray(plabels, dtype=np.int32)
    gl = np.ascontiguousarray(glabels, dtype=np.int32)
    out = np.zeros(1, dtype=np.uint64)
    rc = _load().oracle_count_labeled(adj.shape[0], _p(adj), _p(pl), g.n, _p(g.row_ptr), _p(g.col), _p(gl),
                                      threads or default_threads(), _p(out))
    if rc:
        raise ValueError(f"oracle_count_labeled failed ({rc})")
    return int(out[0])


def degree_relabel(g):
    """Relabel vertices by non-increasing degree, ties by smaller id (the
    definition of the library's degree order). Returns (graph, new2old)."""
    deg = np.diff(g.row_ptr)
    new2old = np.lexsort((np.arange(g.n), -deg)).astype(np.int32)
    old2new = np.empty(g.n, dtype=np.int32)
    old2new[new2old] = np.arange(g.n, dtype=np.int32)
    src = np.repeat(np.arange(g.n, dtype=np.int32), deg)
    return build_csr(g.n, old2new[src], old2new[g.col]), new2old


def triangles(g, threads=None):
    """Unordered triangles of the graph."""
    out = np.zeros(1, dtype=np.uint64)
    rc = _load().oracle_triangles(g.n, _p(g.row_ptr), _p(g.col), threads or default_threads(), _p(out))
    if rc:
        raise ValueError(f"oracle_triangles failed ({rc})")
    return int(out[0])


# ---------------------------------------------------------------- directed

class DCsr:
    """Directed simple graph: sorted out-lists and in-lists."""

    def __init__(self, n, out_ptr, out_col, in_ptr, in_col):
        self.n = n
        self.out_ptr, self.out_col = out_ptr, out_col
        self.in_ptr, self.in_col = in_ptr, in_col

    @property
    def narcs(self):
        return int(self.out_ptr[-1])


def build_dcsr(n, src, dst):
    """Arcs src[i] -> dst[i]: loops dropped, repeated arcs kept once."""
    src = np.ascontiguousarray(src, dtype=np.int32)
    dst = np.ascontiguousarray(dst, dtype=np.int32)
    m = len(src)
    out_ptr = np.zeros(n + 1, dtype=np.int64)
    in_ptr = np.zeros(n + 1, dtype=np.int64)
    out_col = np.zeros(max(1, m), dtype=np.int32)
    in_col = np.zeros(max(1, m), dtype=np.int32)
    narcs = np.zeros(1, dtype=np.int64)
    rc = _load().oracle_build_dcsr(n, m, _p(src), _p(dst), _p(out_ptr), _p(out_col), _p(in_ptr), _p(in_col),
                                   _p(narcs))
    if rc:
        raise ValueError(f"oracle_build_dcsr failed ({rc})")
    a = int(narcs[0])
    return DCsr(n, out_ptr, out_col[:a].copy(), in_ptr, in_col[:a].copy())


def _dadj(adj):
    adj = np.ascontiguousarray(adj, dtype=np.uint8)
    if adj.ndim != 2 or adj.shape[0] != adj.shape[1]:
        raise ValueError("adjacency must be k x k")
    return adj


def aut_count_directed(adj):
    """Arc-preserving permutations of a directed pattern."""
    adj = _dadj(adj)
    out = np.zeros(1, dtype=np.uint64)
    rc = _load().oracle_aut_count_directed(adj.shape[0], _p(adj), _p(out))
    if rc:
        raise ValueError(f"oracle_aut_count_directed failed ({rc})")
    return int(out[0])


def count_maps_directed(adj, dg, order=None, restrictions=(), root_begin=0, root_end=None, threads=None):
    """Injective arc-preserving maps (obeying the restrictions, with the
    first searched vertex's image in [root_begin, root_end))."""
    adj = _dadj(adj)
    k = adj.shape[0]
    o = None if order is None else np.ascontiguousarray(order, dtype=np.int32)
    res = np.ascontiguousarray(np.array(restrictions, dtype=np.int32).reshape(-1, 2))
    nres = res.shape[0]
    if nres == 0:
        res = np.zeros((1, 2), dtype=np.int32)
    hi = np.zeros(1, dtype=np.uint64)
    lo = np.zeros(1, dtype=np.uint64)
    dummy = np.zeros(1, dtype=np.int32)
    rc = _load().oracle_count_directed(k, _p(adj), None if o is None else _p(o), nres, _p(res), dg.n,
                                       _p(dg.out_ptr), _p(dg.out_col if dg.narcs else dummy),
                                       _p(dg.in_ptr), _p(dg.in_col if dg.narcs else dummy),
                                       root_begin, dg.n if root_end is None else root_end,
                                       threads or default_threads(), _p(hi), _p(lo))
    if rc:
        raise ValueError(f"oracle_count_directed failed ({rc})")
    return (int(hi[0]) << 64) | int(lo[0])


def count_directed(adj, dg, threads=None):
    """count(P, G) = arc-preserving injective maps / |Aut(P)|."""
    maps = count_maps_directed(adj, dg, threads=threads)
    aut = aut_count_directed(adj)
    if maps % aut:
        raise AssertionError("map count is not a multiple of |Aut(P)|")
    return maps // aut


# ------------------------------------------------------ inclusion-exclusion

def iep_total(adj, sched, restrictions, kk, g):
    """Section IV-D on a small graph, in plain Python: enumerate the first
    k - kk searched vertices (edges and the restrictions among them
    checked), then, instead of looping over the last kk vertices (pairwise
    non-adjacent, all their pattern neighbours among the first k - kk),
    count the tuples of distinct vertices from their candidate sets with
    the inclusion-exclusion expansion of ``planner_ref.iep_count``
    (Algorithm 2 for every term). Candidate sets exclude the matched
    vertices. Restrictions that involve a last-kk vertex are dropped, as the
    paper drops them; the caller divides by the multiplicity."""
    from .planner_ref import iep_count
    adj = _adj(adj)
    k = adj.shape[0]
    outer, inner = list(sched[:k - kk]), list(sched[k - kk:])
    for a in inner:
        for b in inner:
            if a != b and adj[a, b]:
                raise ValueError("the last kk searched vertices must be pairwise non-adjacent")
    nbr = [set(g.col[g.row_ptr[v]:g.row_ptr[v + 1]].tolist()) for v in range(g.n)]
    ro = [(a, b) for a, b in restrictions if a in outer and b in outer]
    pos = {v: i for i, v in enumerate(outer)}
    img = {}
    total = 0

    def rec(d):
        nonlocal total
        if d == len(outer):
            used = set(img.values())
            sets = []
            for u in inner:
                cand = None
                for w in range(k):
                    if adj[u, w]:
                        cand = set(nbr[img[w]]) if cand is None else cand & nbr[img[w]]
                sets.append((cand if cand is not None else set(range(g.n))) - used)
            total += iep_count(sets)
            return
        x = outer[d]
        earlier = [w for w in outer[:d] if adj[x, w]]
        cands = set(range(g.n)) if not earlier else set.intersection(*(nbr[img[w]] for w in earlier))
        for v in sorted(cands):
            if v in img.values():
                continue
            if any((a == x and pos[b] < d and not v > img[b]) or (b == x and pos[a] < d and not img[a] > v)
                   for a, b in ro):
                continue
            img[x] = v
            rec(d + 1)
            del img[x]
    rec(0)
    return total

