"""SplitMix64 as a counter-based generator, vectorised in numpy uint64."""

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(counters, seed):
    """Return SplitMix64 outputs for an array of uint64 counters.

    Output ``i`` is the finaliser applied to ``seed + (counters[i] + 1) * golden``,
    which is exactly the i-th value a sequential SplitMix64 seeded with
    ``seed`` would return.
    """
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + (np.asarray(counters, dtype=np.uint64) + np.uint64(1)) * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def stream(seed, start, count):
    """``count`` consecutive SplitMix64 outputs starting at counter ``start``."""
    return splitmix64(np.arange(start, start + count, dtype=np.uint64), seed)


def uniform01(bits):
    """Map uint64 outputs to doubles in [0, 1) using their top 53 bits."""
    return (np.asarray(bits, dtype=np.uint64) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
