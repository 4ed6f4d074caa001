"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This package draws graphs and patterns only. It holds none of the counting
method's arithmetic (no CSR building, no set intersection, no symmetry
breaking), so that the oracle and the CUDA path can both consume its output
without sharing any of the computation they are compared on.

Every random number comes from one counter-based generator, SplitMix64
(Steele, Lea and Flood, "Fast splittable pseudorandom number generators",
OOPSLA 2014), evaluated as ``mix(seed + (i + 1) * 0x9E3779B97F4A7C15)`` for
counter ``i``. It is written out in numpy uint64 arithmetic, so the streams are
identical on every machine and numpy version.
"""

from .rng import splitmix64, uniform01, stream
from .graphs import (
    er_edges,
    rmat_edges,
    chung_lu_edges,
    chung_lu_weights,
    WORKLOADS,
    workload_edges,
)
from .patterns import (
    NAMED_PATTERNS,
    named_pattern,
    random_connected_pattern,
    random_pattern_set,
    is_connected,
    edges_to_adj,
)

__all__ = [
    "splitmix64", "uniform01", "stream",
    "er_edges", "rmat_edges", "chung_lu_edges", "chung_lu_weights",
    "WORKLOADS", "workload_edges",
    "NAMED_PATTERNS", "named_pattern", "random_connected_pattern",
    "random_pattern_set", "is_connected", "edges_to_adj",
]
