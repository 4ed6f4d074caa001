"""The seeded input recipes stay what the measurements were taken on: the
counter-based SplitMix64 reproduces the published reference sequence, and
the workload graphs (built by the oracle's CSR builder from the generated
pairs) keep the sizes the measurements were reported on. CPU only; the
two full-size graphs take about a minute together."""

import numpy as np
import pytest

import oracle
from synth import workload_edges
from synth.rng import splitmix64, stream


def test_splitmix64_reference_sequence():
    # the first outputs of the reference SplitMix64 (Steele, Lea and Flood,
    # OOPSLA 2014) seeded with 1234567, as its C reference prints them
    assert [int(x) for x in stream(1234567, 0, 5)] == [
        6457827717110365317, 3203168211198807973, 9817491932198370423,
        4593380528125082431, 16408922859458223821]
    # counter-based: any window of the stream equals the same slice of a longer one
    assert [int(x) for x in stream(7, 1000, 4)] == [int(x) for x in stream(7, 0, 1004)[1000:]]
    assert int(splitmix64(np.array([3], np.uint64), 7)[0]) == int(stream(7, 3, 1)[0])


def _stats(name):
    n, s, d = workload_edges(name)
    g = oracle.build_csr(n, s, d)
    deg = np.diff(g.row_ptr)
    return n, len(s), int(g.row_ptr[-1]) // 2, int(deg.max()), int((deg == 0).sum()), deg


def test_er2000_recipe():
    n, pairs, m, _, _, _ = _stats("er2000")
    assert (n, pairs, m) == (2000, 20000, 19905)


def test_rmat20_recipe():
    n, pairs, m, dmax, isolated, deg = _stats("rmat20")
    assert (n, pairs, m, dmax, isolated) == (1 << 20, 16 << 20, 15700364, 64790, 402679)
    assert float(np.median(deg[deg > 0])) == 5.0


@pytest.mark.parametrize("name", ["cl4m"])
def test_chung_lu_4m_recipe(name):
    n, pairs, m, dmax, isolated, deg = _stats(name)
    assert (n, pairs, m, dmax, isolated) == (4_000_000, 35_000_000, 34561384, 17689, 66999)
    assert abs(float(deg.mean()) - 17.28) < 0.01
