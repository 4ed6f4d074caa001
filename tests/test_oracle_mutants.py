"""The oracle's pins are strong enough to catch plausible mistakes: each test
here plants one mistake in a copy of ``oracle.c`` (on the CPU), builds it,
and checks that a battery of checks fixed by mathematics or brute force
fails on the mutant while it passes on the real oracle. CPU only."""

import ctypes
import itertools
import math
import os
import subprocess

import numpy as np
import pytest

import oracle
from oracle import planner_ref as pr
from synth import er_edges, named_pattern

SRC = os.path.join(os.path.dirname(os.path.abspath(oracle.__file__)), "oracle.c")

# (name, text in oracle.c, replacement): one plausible mistake each
MUTANTS = [
    ("keeps_self_loops", "if (u == v) continue;", ";"),
    ("keeps_duplicates", "if (i == 0 || key[i] != key[i - 1]) key[out++] = key[i];", "key[out++] = key[i];"),
    ("not_injective", "for (int j = 0; j < d; ++j) if (img[j] == v) return 0;                 /* injective */", ";"),
    ("drops_an_edge_check", "if (!has_edge(w, img[w->chk[d][c]], v)) return 0;                   /* edges */",
     "if (c > 0 && !has_edge(w, img[w->chk[d][c]], v)) return 0;"),
    ("ignores_restrictions", "if (w->res_gt[d][r] ? !(v > o) : !(v < o)) return 0;                /* restriction */",
     ";"),
    ("misses_last_neighbour", "    return lo < w->row_ptr[u + 1] && w->col[lo] == v;",
     "    return lo < w->row_ptr[u + 1] - 1 && w->col[lo] == v;"),
    ("aut_ignores_edges", "                if (adj[a * k + b] && !adj[p[a] * k + p[b]]) ok = 0;\n        c += (uint64_t)ok;",
     "                ;\n        c += (uint64_t)ok;"),
    ("wrong_divisor", "    if (maps % aut) return -3;\n    u128 q = maps / aut;",
     "    u128 q = maps / (aut > 1 ? aut / 2 : aut);"),
    ("triangles_counted_twice", "                    if (c <= b) continue;\n", ""),
    ("ignores_graph_labels", "if (w->glab && w->glab[v] != w->plab[d]) return 0;                     /* label */", ";"),
    ("ignores_the_root_label", "if (w->glab && w->glab[img[0]] != w->plab[0]) continue;", ";"),
    ("root_range_shifted", "img[0] = (int32_t)(w->root_begin + i * w->root_stride);",
     "img[0] = (int32_t)(w->root_begin + i * w->root_stride - (i > 0));"),   # stays in range
    ("entry_range_shifted", "int64_t x = w->entry_begin + i;",
     "int64_t x = w->entry_begin + i - (i > 0 && i + 1 == (long)(w->entry_end - w->entry_begin));"),
    ("entry_row_off_by_one", "if (w->row_ptr[mid] <= e) lo = mid; else hi = mid - 1;",
     "if (w->row_ptr[mid] < e) lo = mid; else hi = mid - 1;"),
    ("entry_skips_depth_one_checks", "if (!admit(w, 1, img, w->col[x])) continue;", ";"),
    ("directed_ignores_arc_direction", "good = w->chk_fwd[d][c] ? arc_present(w, o, v) : arc_present(w, v, o);",
     "good = arc_present(w, o, v) || arc_present(w, v, o);"),
    ("directed_keeps_repeated_arcs", "if (uniq == 0 || fwd[i] != fwd[uniq - 1]) fwd[uniq++] = fwd[i];",
     "fwd[uniq++] = fwd[i];"),
    ("listing_not_injective", "        for (int j = 0; j < d && ok; ++j) if (img[j] == v) ok = 0;\n        for (int c = 0; c < w->nchk[d] && ok; ++c)\n            if (!has_edge(w, img[w->chk[d][c]], v)) ok = 0;\n        for (int r = 0; r < w->nres[d] && ok; ++r) {\n            int32_t o",
     "        for (int c = 0; c < w->nchk[d] && ok; ++c)\n            if (!has_edge(w, img[w->chk[d][c]], v)) ok = 0;\n        for (int r = 0; r < w->nres[d] && ok; ++r) {\n            int32_t o"),
]


def complete(n):
    s, d = zip(*itertools.combinations(range(n), 2))
    return oracle.build_csr(n, np.array(s, np.int32), np.array(d, np.int32))


def bipartite(a, b):
    s, d = zip(*[(i, a + j) for i in range(a) for j in range(b)])
    return oracle.build_csr(a + b, np.array(s, np.int32), np.array(d, np.int32))


def dense(g):
    m = np.zeros((g.n, g.n), np.uint8)
    for v in range(g.n):
        m[v, g.col[g.row_ptr[v]:g.row_ptr[v + 1]]] = 1
    return m


def brute_maps(p, gadj):
    k, n = p.shape[0], gadj.shape[0]
    pe = [(x, y) for x in range(k) for y in range(k) if p[x, y]]
    return sum(1 for t in itertools.permutations(range(n), k) if all(gadj[t[x], t[y]] for x, y in pe))


def battery():
    """Checks fixed by mathematics or brute force; returns the failed ones."""
    failed = []

    def check(name, ok):
        if not ok:
            failed.append(name)
    try:
        # CSR of a tiny list with a self loop and duplicates, worked by hand
        g = oracle.build_csr(3, np.array([0, 1, 1, 1, 0], np.int32), np.array([1, 0, 1, 2, 1], np.int32))
        check("csr", list(g.row_ptr) == [0, 1, 3, 4] and list(g.col) == [1, 0, 2, 1])
        check("aut", oracle.aut_count(named_pattern("c4")) == 8 and oracle.aut_count(named_pattern("house")) == 2)
        k7 = complete(7)
        check("cliques", oracle.count(named_pattern("k4"), k7) == math.comb(7, 4))
        check("c4_bipartite", oracle.count(named_pattern("c4"), bipartite(3, 4)) == math.comb(3, 2) * math.comb(4, 2))
        check("triangles", oracle.triangles(k7) == math.comb(7, 3))
        s, d = er_edges(9, 24, seed=4)
        small = oracle.build_csr(9, s, d)
        house = named_pattern("house")
        check("brute_force", oracle.count_maps(house, small) == brute_maps(house, dense(small)))
        s, d = er_edges(30, 140, seed=2)
        g30 = oracle.build_csr(30, s, d)
        adj = house.tolist()
        sched = pr.efficient_schedules(adj)[0][0]
        rs = pr.restriction_sets(adj)[0]
        restricted = oracle.count_restricted(house, sched, rs, g30)
        check("restricted_times_aut", restricted * 2 == oracle.count_maps(house, g30))
        _, listed = oracle.list_restricted(house, sched, rs, g30)
        check("listing", listed == restricted)
        # entry ranges: one root's row gives that root's count; cuts of all
        # entries add up to the whole restricted count
        r = int(np.argmax(np.diff(g30.row_ptr)))
        row = oracle.count_restricted_entries(house, sched, rs, g30, g30.row_ptr[r], g30.row_ptr[r + 1])
        check("entry_row", row == oracle.count_restricted(house, sched, rs, g30, root_begin=r, root_end=r + 1))
        cuts = [0, 3, 50, 51, 97, int(g30.row_ptr[-1])]
        parts = sum(oracle.count_restricted_entries(house, sched, rs, g30, a, b) for a, b in zip(cuts, cuts[1:]))
        check("entry_cuts", parts == restricted)
        # a restriction acting at the second searched vertex: triangles with
        # id(0) > id(1) > id(2) in search order (0, 1, 2), over entry cuts
        tri = named_pattern("triangle")
        tparts = sum(oracle.count_restricted_entries(tri, (0, 1, 2), [(0, 1), (1, 2)], g30, a, b)
                     for a, b in zip(cuts, cuts[1:]))
        check("entry_restriction", tparts == oracle.triangles(g30))
        a, b = 3, 4
        gl = [0] * a + [1] * b
        check("labels", oracle.count_labeled(named_pattern("c4"), [0, 1, 0, 1], bipartite(a, b), gl)
              == math.comb(a, 2) * math.comb(b, 2)
              and oracle.count_labeled(named_pattern("c4"), [0, 0, 1, 1], bipartite(a, b), gl) == 0)
        # path a-b-c labelled 0, 1, 1 in K4 labelled 0, 1, 1, 1: the root is
        # the one label-0 vertex, then 3 x 2 ordered label-1 vertices
        path3 = np.array([[0, 1, 0], [1, 0, 1], [0, 1, 0]], np.uint8)
        check("root_label", oracle.count_labeled(path3, [0, 1, 1], complete(4), [0, 1, 1, 1]) == 6)
        # directed: hand-worked lists, a transitive tournament, a complete digraph
        dg = oracle.build_dcsr(3, np.array([0, 1, 1, 0], np.int32), np.array([1, 0, 2, 1], np.int32))
        check("dcsr", list(dg.out_ptr) == [0, 1, 3, 3] and list(dg.out_col) == [1, 0, 2])
        cyc3 = np.zeros((3, 3), np.uint8)
        cyc3[0, 1] = cyc3[1, 2] = cyc3[2, 0] = 1
        ff = np.zeros((3, 3), np.uint8)
        ff[0, 1] = ff[0, 2] = ff[1, 2] = 1
        t6 = [(i, j) for i in range(6) for j in range(i + 1, 6)]
        T = oracle.build_dcsr(6, np.array([a for a, _ in t6], np.int32), np.array([b for _, b in t6], np.int32))
        check("tournament", oracle.count_directed(cyc3, T) == 0 and oracle.count_directed(ff, T) == 20)
    except Exception as e:              # a mutant may also break an internal consistency check
        failed.append(f"raised {type(e).__name__}")
    return failed


def test_real_oracle_passes_the_battery():
    assert battery() == []


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_mutant_is_caught(tmp_path, name, old, new):
    src = open(SRC).read()
    assert src.count(old) == 1, f"{name}: the planted text must occur exactly once"
    (tmp_path / "oracle.c").write_text(src.replace(old, new))
    (tmp_path / "oracle.h").write_text(open(os.path.join(os.path.dirname(SRC), "oracle.h")).read())
    so = tmp_path / "libmutant.so"
    subprocess.check_call(["gcc", "-O1", "-std=c11", "-w", "-fPIC", "-shared", "-pthread",
                           str(tmp_path / "oracle.c"), "-o", str(so)])
    saved = oracle._lib
    oracle._lib = oracle.configure(ctypes.CDLL(str(so)))
    try:
        failed = battery()
    finally:
        oracle._lib = saved
    assert failed, f"mutant {name} passed every check"
