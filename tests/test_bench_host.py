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
