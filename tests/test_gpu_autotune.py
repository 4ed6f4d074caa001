"""Autotuner: every launch configuration it tries gives the same counts,
and the chosen configuration reproduces the oracle's count."""

import json

import pytest

import oracle
from synth import named_pattern, workload_edges

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2009_10955_gb300 import native
    N = native()
    graphs = {}
    for name in ("rmat10", "er2000"):
        n, s, d = workload_edges(name)
        graphs[name] = (N.gp_graph_create_edges(s, d, n, N.GP_DEGREE_ORDER), oracle.build_csr(n, s, d))
    return N, graphs


def test_knobs_do_not_change_counts(env):
    N, graphs = env
    for gname, pname in (("rmat10", "triangle"), ("rmat10", "k4"), ("er2000", "house"), ("er2000", "k4")):
        g, ref = graphs[gname]
        adj = named_pattern(pname)
        sc = N.gp_schedule(N.gp_pattern_create(adj), g)
        expect = oracle.count(adj, ref)
        for bps in (2, 3, 4):
            for lane_work in (1, 64, 100000):
                for flags in (0, N.GP_COUNT_NO_CORE):
                    for chunk in (0, 1, 7):
                        for split in (1, 5):
                            o = N.make_opts(blocks_per_sm=bps, lane_work=lane_work, flags=flags, chunk=chunk,
                                            split=split)
                            assert N.gp_count(g, sc, 0, o) == (N.GP_OK, expect), \
                                (pname, bps, lane_work, flags, chunk, split)


def test_tune_returns_and_caches(env, tmp_path):
    from paper_2009_10955_gb300 import autotune
    N, graphs = env
    g, ref = graphs["rmat10"]
    adj = named_pattern("k4")
    sc = N.gp_schedule(N.gp_pattern_create(adj), g)
    cache = str(tmp_path / "tune.json")
    space = {"blocks_per_sm": [2, 4], "lane_work": [64, 192], "core": [True, False], "chunk": [0], "split": [1]}
    best, table = autotune.tune(g, sc, 0, space=space, windows=16, width=256, cache_path=cache)
    assert len(table) == 8 and best in [c for c, _ in table]
    best2, _ = autotune.tune(g, sc, 0, space=space, cache_path=cache)
    assert best2 == best
    assert json.load(open(cache))
    assert N.gp_count(g, sc, 0, autotune.opts_for(best)) == (N.GP_OK, oracle.count(adj, ref))


@pytest.mark.parametrize("gname,pname", [("rmat10", "house"), ("er2000", "k4"), ("rmat10", "star5")])
def test_plan_choice_by_sample(env, gname, pname, tmp_path):
    """The sampled plan choice: every candidate (top plans and their mirror
    images, with inclusion-exclusion where it applies) is timed, and the
    chosen plan's whole count equals the oracle's; a second call takes the
    cached choice."""
    from paper_2009_10955_gb300 import autotune
    N, graphs = env
    g, ref = graphs[gname]
    adj = named_pattern(pname)
    cache = str(tmp_path / "plans.json")
    sched, table = autotune.choose_plan(g, adj, top_k=3, windows=16, width=8, cache_path=cache)
    assert len(table) >= 2 and all(t is not None for *_, t in table)
    mirrored = {(tuple(o), tuple(map(tuple, r))) for o, r, _, _ in table}
    for o, r, _, _ in table:
        assert (tuple(o), tuple((b, a) for a, b in r)) in mirrored
    if pname in ("house", "star5"):        # both forms of plans that qualify for inclusion-exclusion
        assert {kk > 0 for _, _, kk, _ in table} == {True, False}
    if pname.startswith("star"):       # closed form: a centre and L of its neighbours
        from math import comb
        import numpy as np
        expect = sum(comb(int(d), adj.shape[0] - 1) for d in np.diff(ref.row_ptr))
    else:
        expect = oracle.count(adj, ref)
    assert N.gp_count(g, sched) == (N.GP_OK, expect)
    again, table2 = autotune.choose_plan(g, adj, top_k=3, windows=16, width=8, cache_path=cache)
    assert table2 == json.loads(json.dumps(table)) and again.get(0)[:2] == sched.get(0)[:2]
    assert N.gp_count(g, again) == (N.GP_OK, expect)
