"""The product path and the oracle are independent: the package imports
nothing from oracle/, its C/CUDA sources include nothing from there, the
library exports no oracle symbol, and the oracle includes nothing of the
library. CPU only."""

import glob
import os
import re
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2009_10955_gb300")


def test_package_modules_do_not_import_the_oracle():
    code = ("import sys; sys.path.insert(0, %r)\n"
            "import paper_2009_10955_gb300, paper_2009_10955_gb300._native, paper_2009_10955_gb300.autotune\n"
            "import paper_2009_10955_gb300.serve, paper_2009_10955_gb300.shard, paper_2009_10955_gb300.build\n"
            "paper_2009_10955_gb300.native()\n"
            "print(sorted(m for m in sys.modules if m == 'oracle' or m.startswith('oracle.')))\n") % ROOT
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, check=True)
    assert out.stdout.strip() == "[]"


def test_sources_share_nothing():
    pat_py = re.compile(r"^\s*(from\s+oracle\b|import\s+oracle\b)", re.M)
    for f in glob.glob(os.path.join(PKG, "*.py")):
        assert not pat_py.search(open(f).read()), f
    for f in glob.glob(os.path.join(PKG, "csrc", "*")):
        text = open(f).read()
        assert not re.search(r'#\s*include\s*[<"][^>"]*oracle', text), f
    for f in glob.glob(os.path.join(ROOT, "oracle", "*")):
        if f.endswith((".c", ".h", ".py")):
            text = open(f).read()
            assert "graphpi.h" not in text and "paper_2009_10955_gb300" not in text, f


def test_library_exports_no_oracle_symbol():
    from paper_2009_10955_gb300 import native
    lib = native().lib()
    path = lib._name
    syms = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True, check=True).stdout
    assert "oracle" not in syms


def test_no_cpu_fallback_without_a_device():
    """Without a usable CUDA device the counting path fails loudly with
    GP_ERR_CUDA; nothing is computed on the host instead."""
    import numpy as np
    import pytest
    import torch
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    from paper_2009_10955_gb300 import native
    N = native()
    with pytest.raises(N.GraphPiError) as e:
        N.gp_graph_create_edges(np.array([0, 1], np.int32), np.array([1, 2], np.int32), 3, N.GP_DEGREE_ORDER)
    assert e.value.status == N.GP_ERR_CUDA
