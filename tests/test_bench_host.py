"""Host helpers of the benchmark (CPU): the code-only source hash that keys
recorded DRAM traffic ignores comments and whitespace but not code."""

import importlib.util
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def bench():
    spec = importlib.util.spec_from_file_location("bench_host_under_test", os.path.join(ROOT, "bench.py"))
    b = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(b)
    return b


def test_code_only_drops_comments_keeps_literals():
    b = bench()
    src = 'int a = 1; // note\n/* block\n comment */ const char* s = "x // y /* z */";\nchar q = \'/\';  int  c;'
    assert b._code_only(src) == 'int a = 1; const char* s = "x // y /* z */"; char q = \'/\'; int c;'
    assert b._code_only("a /* it's */ b // don't\nc") == "a b c"
    assert b._code_only("x = 1;") != b._code_only("x = 2;")
    assert b._code_only("x  =\n  1;") == b._code_only("x = 1;")


def test_escaped_quote_inside_literal():
    b = bench()
    assert b._code_only('s = "a\\"b // c"; // d') == 's = "a\\"b // c";'


def test_degree_strata_partition_the_degree_order():
    """Strata of degree [2^i, 2^(i+1)) are contiguous id ranges of the
    degree-ordered graph, in order, covering every non-isolated vertex."""
    import numpy as np
    import oracle
    from synth import workload_edges
    b = bench()
    n, s, d = workload_edges("rmat12")
    g, _ = oracle.degree_relabel(oracle.build_csr(n, s, d))
    deg = np.diff(g.row_ptr)
    strata = b.degree_strata(n, s, d)
    assert strata[0][0] == 0
    for (a0, b0, _), (a1, _, _) in zip(strata, strata[1:]):
        assert b0 == a1
    assert strata[-1][1] == int(np.count_nonzero(deg))
    for a, e, lo in strata:
        assert a < e and lo & (lo - 1) == 0
        assert deg[a:e].min() >= lo and deg[a:e].max() < 2 * lo


def test_task_sampler_is_stratified():
    """One window per equal slice of the task space, inside its slice, all
    windows disjoint and of the requested width; a space smaller than the
    sample is taken whole."""
    from paper_2009_10955_gb300.autotune import sample_ranges
    nnz, windows, width = 1_000_003, 97, 50
    r = sample_ranges(nnz, windows, width, seed=5)
    step = nnz // windows
    assert len(r) == windows
    for i, (a, e) in enumerate(r):
        assert e - a == width and i * step <= a and e <= (i + 1) * step
    assert sample_ranges(100, 10, 20) == [(0, 100)]
    assert sample_ranges(nnz, windows, width, seed=5) == r and sample_ranges(nnz, windows, width, seed=6) != r


def test_busy_cycle_projection():
    """The projection spreads a sample's busy warp cycles, scaled to all
    tasks, over the launch's warps at the clock rate."""
    from paper_2009_10955_gb300.autotune import project_s
    assert project_s((2.07e9 * 1000, 1000), 10, 100) == 10.0
    assert project_s((5, 0), 10, 100) is None and project_s((5, 8), 0, 100) is None


def test_alu_peak_from_unit_counts():
    b = bench()
    peak, src = b.alu_peak_gops(152)
    assert "152 SMs" in src
    mhz = float(src.split(" MHz")[0].split("x")[-1])
    assert abs(peak - 152 * 4 * 16 * mhz * 1e-3) < 1e-6


def test_plan_mode_covers_every_named_pattern():
    """bench.py --mode plan (host planning time): one row per named pattern,
    with the automorphism count of the oracle's planner restatement."""
    from oracle import planner_ref as pr
    from synth import named_pattern
    from synth.patterns import NAMED_PATTERNS
    out = bench().plan_bench(repeats=1)
    assert set(out["patterns"]) == set(NAMED_PATTERNS)
    for name, row in out["patterns"].items():
        assert row["restriction_sets"] > 0 and row["schedules"] > 0 and row["plans"] >= 1
        assert row["plan_ms"] >= 0.0
        if row["k"] <= 6:
            assert row["aut"] == len(pr.automorphisms(named_pattern(name).tolist()))


def test_clock_sampler_summary():
    """The clocks record of the line: median SM clock under load, the maximum,
    and every throttle reason seen active in any sample."""
    b = bench()

    class FakeProc:
        def terminate(self):
            pass

        def wait(self, timeout=None):
            return 0

    cs = object.__new__(b.ClockSampler)
    cs.proc, cs.uuid = FakeProc(), "GPU-fake"
    cs.rows = [["2070", "2070", "900.5", "0x0", "Not Active", "Not Active", "Not Active", "Not Active"],
               ["1965", "2070", "1390.0", "0x4", "Not Active", "Not Active", "Not Active", "Active"],
               ["2070", "2070", "1000.0", "0x0", "Not Active", "Not Active", "Not Active", "Not Active"],
               ["[N/A]", "2070", "1000.0", "0x0", "Not Active", "Active", "Not Active", "Not Active"]]
    out = cs.stop()
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0 and out["samples"] == 4
    assert out["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]


def test_both_arms_report_one_config():
    """The reference arm's config is the workload's, built by the same
    function the GPU arm uses, with sizes from the oracle's CSR of the same
    pairs (which the GPU graph build matches bit for bit)."""
    import argparse
    import oracle
    from synth import workload_edges
    import bench as b                 # importable by name: the oracle runs in spawned children
    a = argparse.Namespace(workload="er2000", patterns=None, steps=1, warmup=0, gpus=1)
    out = b.reference_arm(a)
    n, s, d = workload_edges("er2000")
    g = oracle.build_csr(n, s, d)
    import numpy as np
    expect = b.workload_config("er2000", "er2000", n, int(g.row_ptr[-1]) // 2, int(np.diff(g.row_ptr).max()),
                               ["house"])
    assert out["config"] == expect
    assert set(expect) == {"workload", "graph", "n", "m_undirected", "max_deg", "patterns", "l2"}
    assert out["impl"] == "reference" and out["e2e"]["value"] == out["value"]


def test_driver_command_lines_parse(monkeypatch):
    """The command lines the benchmark is launched with parse, with N = 1
    and a few-minute run as the defaults."""
    import sys
    b = bench()
    monkeypatch.setattr(sys, "argv", ["bench.py"])
    a = b.parse()
    assert (a.gpus, a.impl, a.workload, a.mode) == (1, "gb300", "rmat20", "count") and a.warmup >= 3
    for argv in (["--gpus", "1", "--steps", "20", "--warmup", "5"],
                 ["--impl", "reference", "--gpus", "2", "--steps", "20", "--warmup", "5"],
                 ["--workload", "cl4m", "--steps", "2"], ["--mode", "plan"], ["--mode", "iep"]):
        monkeypatch.setattr(sys, "argv", ["bench.py"] + argv)
        b.parse()
