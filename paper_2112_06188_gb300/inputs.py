"""Seeded synthetic workloads shaped like the paper's experiments (Sec. VI).

This module holds no arithmetic of the method: it only draws points, ids and
queries.  It is shared by the tests, the benchmark and the CPU oracle runs, so
both sides of every parity check see the same inputs.

The paper's datasets (Uniform in a hypercube of side sqrt(n), Gan-Tao
VisualVar, three real sets) are not available; these stand in for them:

* uniform integer points on the 2^20 grid (stand-in for Uniform),
* a mixture of Gaussian clusters with log-uniform widths (stand-in for the
  variable-density VisualVar set),
* delete batches drawn uniformly without replacement from the live ids,
* queries drawn uniformly, or as points of the live set (k-NN graph style).
"""
import numpy as np

GRID = 1 << 20          # coordinates live on [0, 2^20)


def uniform_points(n, dim, seed):
    rng = np.random.default_rng(seed)
    return rng.integers(0, GRID, size=(n, dim), dtype=np.int32)


def gaussian_clusters(n, dim, seed, n_clusters=100, sigma_lo=2.0 ** 8, sigma_hi=2.0 ** 16):
    """Each point picks a cluster uniformly; coordinates round(centre + sigma*N(0,1))
    clipped to the grid; centres uniform, sigma log-uniform in [sigma_lo, sigma_hi]."""
    rng = np.random.default_rng(seed)
    centres = rng.uniform(0, GRID, size=(n_clusters, dim))
    sigma = np.exp(rng.uniform(np.log(sigma_lo), np.log(sigma_hi), size=n_clusters))
    which = rng.integers(0, n_clusters, size=n)
    out = np.empty((n, dim), dtype=np.int32)
    chunk = 1 << 22
    for a in range(0, n, chunk):
        b = min(n, a + chunk)
        w = which[a:b]
        x = centres[w] + sigma[w, None] * rng.standard_normal((b - a, dim))
        out[a:b] = np.clip(np.rint(x), 0, GRID - 1).astype(np.int32)
    return out


def duplicate_heavy_points(n, dim, seed, distinct=7):
    """Many exactly repeated coordinates: stresses ties in splits and distances."""
    rng = np.random.default_rng(seed)
    base = rng.integers(0, GRID, size=(distinct, dim), dtype=np.int32)
    return base[rng.integers(0, distinct, size=n)]


def sample_ids(live_ids, count, seed):
    """`count` distinct ids drawn uniformly from `live_ids`."""
    rng = np.random.default_rng(seed)
    live_ids = np.asarray(live_ids)
    count = min(count, len(live_ids))
    return rng.choice(live_ids, size=count, replace=False).astype(np.int32)


def queries_from(points, m, seed):
    """m rows of `points` drawn uniformly with replacement."""
    rng = np.random.default_rng(seed)
    return np.ascontiguousarray(points[rng.integers(0, len(points), size=m)])


class LiveSet:
    """Host-side record of which ids are live and where their coordinates are."""

    def __init__(self, dim):
        self.dim = dim
        self.coords = np.empty((0, dim), dtype=np.int32)
        self.alive = np.zeros(0, dtype=bool)

    def insert(self, pts):
        first = len(self.alive)
        self.coords = np.concatenate([self.coords, np.asarray(pts, np.int32).reshape(-1, self.dim)])
        self.alive = np.concatenate([self.alive, np.ones(len(pts), dtype=bool)])
        return np.arange(first, first + len(pts), dtype=np.int32)

    def erase(self, ids):
        ids = np.asarray(ids, dtype=np.int64)
        ok = (ids >= 0) & (ids < len(self.alive))
        ids = np.unique(ids[ok])
        n = int(self.alive[ids].sum())
        self.alive[ids] = False
        return n

    def live_ids(self):
        return np.flatnonzero(self.alive).astype(np.int32)

    def live_points(self):
        ids = self.live_ids()
        return self.coords[ids], ids


def config_small_sequence(seed=1, dim=2, n0=65536, n_ins=8, ins=8192, n_del=4, dele=8192,
                          m=4096):
    """The plain small workload: build n0 uniform 2-D points, n_ins insert batches,
    n_del delete batches of live ids, and m uniform queries after every batch.
    Yields ("insert", pts) / ("erase", ids) / ("knn", queries) in order."""
    rng = np.random.default_rng(seed)
    live = LiveSet(dim)

    def pts(n):
        return rng.integers(0, GRID, size=(n, dim), dtype=np.int32)

    def qs():
        return rng.integers(0, GRID, size=(m, dim), dtype=np.int32)

    p = pts(n0)
    live.insert(p)
    yield "insert", p
    yield "knn", qs()
    for _ in range(n_ins):
        p = pts(ins)
        live.insert(p)
        yield "insert", p
        yield "knn", qs()
    for _ in range(n_del):
        ids = rng.choice(live.live_ids(), size=min(dele, int(live.alive.sum())),
                         replace=False).astype(np.int32)
        live.erase(ids)
        yield "erase", ids
        yield "knn", qs()
