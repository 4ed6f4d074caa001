"""Seeded edge-list generators for the synthetic data graphs.

Each generator returns the raw sampled pairs ``(src, dst)`` as int32 arrays.
Self loops and duplicate pairs are left in on purpose: removing them is the
graph-build step of the counting path (and, separately, of the oracle).

Workload shapes stand in for the paper's SNAP graphs (Table I), which are not
available here:

* ``er2000``: G(n=2000, m=20000) sampled pairs, seed 1 (Wiki-Vote scale);
* ``rmat20``: R-MAT scale 20, edge factor 16, a/b/c/d = .57/.19/.19/.05,
  seed 2 (Patents/MiCo-like degree skew);
* ``cl4m``: Chung-Lu, 4,000,000 vertices, 35,000,000 sampled pairs, degree
  exponent 2.1, expected maximum degree 20,000, seed 3 (LiveJournal-like,
  4.0M vertices / 34.7M edges).
"""

import numpy as np

from .rng import splitmix64, stream, uniform01


def er_edges(n, m, seed):
    """G(n, m): ``m`` independent uniform ordered pairs over ``[0, n)``.

    Counter ``2i`` draws the source of pair ``i`` and ``2i + 1`` its target.
    """
    u = uniform01(stream(seed, 0, 2 * m))
    pairs = np.minimum((u * n).astype(np.int64), n - 1).reshape(m, 2)
    return pairs[:, 0].astype(np.int32), pairs[:, 1].astype(np.int32)


def rmat_edges(scale, edge_factor, a, b, c, seed, chunk=1 << 22):
    """R-MAT (Chakrabarti, Zhan and Faloutsos, SDM 2004) without noise.

    ``edge_factor * 2**scale`` pairs. Pair ``e`` descends ``scale`` levels of
    the recursive adjacency-matrix split, most significant bit first; level
    ``l`` uses counter ``e * scale + l``: below ``a`` picks the top-left
    quadrant, below ``a + b`` top-right, below ``a + b + c`` bottom-left,
    otherwise bottom-right. No label permutation is applied.
    """
    m = edge_factor << scale
    src = np.empty(m, dtype=np.int32)
    dst = np.empty(m, dtype=np.int32)
    ab, abc = a + b, a + b + c
    for lo in range(0, m, chunk):
        hi = min(m, lo + chunk)
        e = np.arange(lo, hi, dtype=np.uint64)
        s = np.zeros(hi - lo, dtype=np.int64)
        d = np.zeros(hi - lo, dtype=np.int64)
        for level in range(scale):
            u = uniform01(splitmix64(e * np.uint64(scale) + np.uint64(level), seed))
            right = ((u >= a) & (u < ab)) | (u >= abc)
            down = u >= ab
            s = (s << 1) | down
            d = (d << 1) | right
        src[lo:hi] = s
        dst[lo:hi] = d
    return src, dst


def chung_lu_weights(n, gamma, w_max, w_mean):
    """Expected degrees ``w_i = C * (i + i0) ** (-1 / (gamma - 1))``.

    ``i0`` is found by bisection so that ``w_0 / mean(w) = w_max / w_mean``;
    ``C`` then scales the mean to ``w_mean``. Vertex 0 has the largest weight.
    """
    expo = -1.0 / (gamma - 1.0)
    i = np.arange(n, dtype=np.float64)
    target = w_max / w_mean

    def ratio(i0):
        w = (i + i0) ** expo
        return w[0] / w.mean()

    lo, hi = 1e-6, float(n)
    for _ in range(200):
        mid = np.sqrt(lo * hi)
        if ratio(mid) > target:
            lo = mid
        else:
            hi = mid
    w = (i + np.sqrt(lo * hi)) ** expo
    return w * (w_mean / w.mean())


def chung_lu_edges(n, m, gamma, w_max, w_mean, seed, chunk=1 << 22):
    """Chung-Lu: ``m`` pairs whose endpoints are drawn independently with
    probability proportional to ``chung_lu_weights``.

    Endpoints are sampled by inverse CDF (a binary search in the cumulative
    weights). Counter ``2e`` draws the source of pair ``e``, ``2e + 1`` its
    target.
    """
    w = chung_lu_weights(n, gamma, w_max, w_mean)
    cdf = np.cumsum(w)
    cdf /= cdf[-1]
    src = np.empty(m, dtype=np.int32)
    dst = np.empty(m, dtype=np.int32)
    for lo in range(0, m, chunk):
        hi = min(m, lo + chunk)
        u = uniform01(stream(seed, 2 * lo, 2 * (hi - lo))).reshape(-1, 2)
        v = np.minimum(np.searchsorted(cdf, u, side="right"), n - 1)
        src[lo:hi] = v[:, 0]
        dst[lo:hi] = v[:, 1]
    return src, dst


# name -> (vertex count, thunk returning (src, dst)). Down-scaled members of
# the same families serve the parity tests.
WORKLOADS = {
    "er2000": (2000, lambda: er_edges(2000, 20000, seed=1)),
    "rmat20": (1 << 20, lambda: rmat_edges(20, 16, 0.57, 0.19, 0.19, seed=2)),
    "cl4m": (4_000_000, lambda: chung_lu_edges(4_000_000, 35_000_000, 2.1, 20000.0, 17.5, seed=3)),
}
for _s in range(8, 20):
    WORKLOADS[f"rmat{_s}"] = (1 << _s, (lambda s: lambda: rmat_edges(s, 16, 0.57, 0.19, 0.19, seed=2))(_s))
for _n in (10_000, 100_000, 1_000_000):
    # same shape as cl4m: mean 17.5, max scaled like sqrt(n) from 20K at 4M
    WORKLOADS[f"cl{_n}"] = (
        _n,
        (lambda n: lambda: chung_lu_edges(
            n, int(n * 17.5 / 2), 2.1, 20000.0 * np.sqrt(n / 4_000_000), 17.5, seed=3))(_n),
    )


def workload_edges(name):
    """Return ``(n, src, dst)`` for a named workload."""
    n, thunk = WORKLOADS[name]
    src, dst = thunk()
    return n, src, dst
