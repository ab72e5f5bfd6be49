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


class ForestsWorkload:
    """Many independent forests of uneven sizes: nf forests with sizes
    log-uniform in [lo, hi] and dimension drawn from `dims`, uniform grid
    points.  Step s gives every forest an insert batch of 5-20% of its initial
    size, then a delete batch of 2-10% of its live ids, then k-NN for 1-5k
    queries drawn from its live set (sizes drawn per forest and step)."""

    def __init__(self, nf=512, lo=1_000, hi=200_000, dims=(2, 3), seed=4, q_lo=1000, q_hi=5000):
        self.rng = np.random.default_rng(seed)
        r = self.rng
        self.sizes = np.exp(r.uniform(np.log(lo), np.log(hi), size=nf)).astype(np.int64)
        self.dims = [int(d) for d in r.choice(dims, size=nf)]
        self.q_lo, self.q_hi = q_lo, q_hi
        self.initial = [r.integers(0, GRID, size=(int(n), d), dtype=np.int32)
                        for n, d in zip(self.sizes, self.dims)]
        # live ids per forest, kept as the next id plus a boolean mask
        self.alive = [np.ones(int(n), dtype=bool) for n in self.sizes]
        self.coords = [p.copy() for p in self.initial]

    def step(self):
        """One step's inputs: a list of (insert points, erase ids, queries) per forest."""
        r = self.rng
        out = []
        for i, d in enumerate(self.dims):
            n_ins = max(1, int(r.uniform(0.05, 0.20) * self.sizes[i]))
            ins = r.integers(0, GRID, size=(n_ins, d), dtype=np.int32)
            self.coords[i] = np.concatenate([self.coords[i], ins])
            self.alive[i] = np.concatenate([self.alive[i], np.ones(n_ins, dtype=bool)])
            live = np.flatnonzero(self.alive[i])
            n_del = max(1, int(r.uniform(0.02, 0.10) * len(live)))
            era = r.choice(live, size=n_del, replace=False).astype(np.int32)
            self.alive[i][era] = False
            live = np.flatnonzero(self.alive[i])
            m = int(r.integers(self.q_lo, self.q_hi + 1))
            q = np.ascontiguousarray(self.coords[i][live[r.integers(0, len(live), size=m)]])
            out.append((ins, era, q))
        return out


def log_uniform_int(rng, lo, hi):
    return int(np.exp(rng.uniform(np.log(lo), np.log(hi))))


class ServeWorkload:
    """A request stream on one growing forest: Poisson arrivals at `rate`
    requests per second; each request is an insert (1k-1M uniform points), an
    erase (1k-500k ids drawn uniformly from the live set) or a k-NN batch (1 to
    100k uniform queries, k drawn from `ks`) in the ratio `mix`; batch sizes
    log-uniform within their ranges.  The initial forest has n0 points; the
    stream ends once the live count reaches n_final or after max_requests."""

    def __init__(self, dim=5, n0=1_000_000, n_final=50_000_000, rate=200.0, seed=5,
                 mix=(4, 1, 5), ins=(1_000, 1_000_000), dele=(1_000, 500_000), knn=(1, 100_000),
                 ks=(1, 5, 10), max_requests=None):
        self.rng = np.random.default_rng(seed)
        self.dim, self.n_final, self.rate = dim, n_final, rate
        self.mix = np.asarray(mix, dtype=np.float64) / sum(mix)
        self.ins, self.dele, self.knn, self.ks = ins, dele, knn, ks
        self.max_requests = max_requests
        self.initial = self.rng.integers(0, GRID, size=(n0, dim), dtype=np.int32)
        self.alive = np.ones(n0, dtype=bool)

    def requests(self):
        """Yields (arrival time in s, kind, payload, k): kind "insert" with points,
        "erase" with ids, "knn" with queries."""
        r, t, count = self.rng, 0.0, 0
        while int(self.alive.sum()) < self.n_final:
            if self.max_requests is not None and count >= self.max_requests:
                return
            t += r.exponential(1.0 / self.rate)
            kind = r.choice(3, p=self.mix)
            if kind == 0:
                n = log_uniform_int(r, *self.ins)
                p = r.integers(0, GRID, size=(n, self.dim), dtype=np.int32)
                self.alive = np.concatenate([self.alive, np.ones(n, dtype=bool)])
                yield t, "insert", p, 0
            elif kind == 1:
                live = np.flatnonzero(self.alive)
                n = min(log_uniform_int(r, *self.dele), len(live))
                ids = r.choice(live, size=n, replace=False).astype(np.int32)
                self.alive[ids] = False
                yield t, "erase", ids, 0
            else:
                m = log_uniform_int(r, *self.knn)
                q = r.integers(0, GRID, size=(m, self.dim), dtype=np.int32)
                yield t, "knn", q, int(r.choice(self.ks))
            count += 1
