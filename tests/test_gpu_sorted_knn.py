"""Row-by-row parity of the k-NN path that large query batches take.

From 2^15 = 32,768 queries per forest on, the CUDA path first puts the
queries in spatial (Morton) order, so that the lanes of a warp walk
neighbouring paths and scan their leaves together -- the path the full-size
workloads run.  These tests compare EVERY row of such calls (ids and squared
distances, bit for bit) with the oracle's kNN_L (Alg. 5), after insert and
erase batches that rebuild trees (Alg. 3, Alg. 4), in 2, 3, 5 and 7
dimensions, through the single-forest call and the batched call (the
allocation-free call is compared with the oracle in test_zz_no_alloc.py).
"""
import numpy as np
import pytest
import torch

from oracle.oracle import OracleForest
from paper_2112_06188_gb300 import inputs
from oracle.threads import oracle_knn

pytestmark = pytest.mark.gpu

SORT_MIN = 1 << 15          # the batch size from which queries run in spatial order


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2112_06188_gb300 import build_lib
    build_lib.build()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def query_mix(live, m, dim, seed):
    """m queries: half of them live points (d2 = 0 hits and dense
    neighbourhoods), half uniform on the grid."""
    lp, _ = live.live_points()
    a = inputs.queries_from(lp, m // 2, seed=seed)
    b = inputs.uniform_points(m - m // 2, dim, seed=seed + 1)
    return np.ascontiguousarray(np.concatenate([a, b]))


def assert_rows(gi, gd, oi, od, what):
    gi, gd = gi.cpu().numpy(), gd.cpu().numpy()
    bad = (gi != oi).any(1) | (gd != od).any(1)
    assert not bad.any(), "%s: %d of %d rows differ (first %d)" % (what, int(bad.sum()), len(bad),
                                                                  int(np.argmax(bad)))


def grow_and_shrink(g, o, live, n0, dim, seed):
    """Yields after two (insert, erase) steps on both forests: the first
    erases 57% of the live points, so every tree falls below half of its
    capacity and is rebuilt (Alg. 4); the second has ragged sizes."""
    rng = np.random.default_rng(seed)
    for ins, frac in ((n0 // 6, 0.57), (n0 // 10 + 517, 0.05)):
        p = rng.integers(0, inputs.GRID, size=(ins, dim), dtype=np.int32)
        g.insert(dev(p))
        o.insert(p)
        live.insert(p)
        lid = live.live_ids()
        era = inputs.sample_ids(lid, int(frac * len(lid)) + 3, seed=seed + ins)
        ne = g.erase(dev(era))
        assert ne == o.erase(era) == live.erase(era)
        assert g.tree_mask() == o.tree_mask() and g.size() == o.size()
        yield


CASES = [
    # dim, n0, queries, k
    (3, 300_000, 65_536, 10),
    (2, 300_000, 65_536, 10),
    (5, 200_000, 40_000, 5),
    (7, 100_000, 40_000, 5),
]


@pytest.mark.parametrize("dim,n0,m,k", CASES)
def test_sorted_path_every_row_matches_oracle(dim, n0, m, k):
    from paper_2112_06188_gb300.forest import Forest
    assert m >= SORT_MIN
    pts = inputs.uniform_points(n0, dim, seed=40 + dim)
    g, o = Forest(dim), OracleForest(dim)
    live = inputs.LiveSet(dim)
    g.insert(dev(pts))
    o.insert(pts)
    live.insert(pts)
    q = query_mix(live, m, dim, seed=50 + dim)
    oi, od = oracle_knn(o, q, k)
    gi, gd = g.knn(dev(q), k)
    assert_rows(gi, gd, oi, od, "after the build")
    for step, _ in enumerate(grow_and_shrink(g, o, live, n0, dim, seed=60 + dim)):
        q = query_mix(live, m, dim, seed=70 + 10 * step + dim)
        oi, od = oracle_knn(o, q, k)
        gi, gd = g.knn(dev(q), k)
        assert_rows(gi, gd, oi, od, "after step %d" % step)
    g.close()


def test_sorted_path_batched_call_matches_oracle():
    """One batched k-NN call over three forests: two of them with more than
    2^15 queries (spatial order), one with fewer (input order), of two
    dimensions; every row against each forest's oracle."""
    from paper_2112_06188_gb300.forest import Forest, knn_batch
    specs = [(3, 150_000, 40_000), (2, 120_000, 50_000), (3, 20_000, 3_000)]
    k = 8
    gs, os_, qs = [], [], []
    for j, (dim, n0, m) in enumerate(specs):
        g, o = Forest(dim), OracleForest(dim)
        live = inputs.LiveSet(dim)
        pts = inputs.uniform_points(n0, dim, seed=80 + j)
        g.insert(dev(pts))
        o.insert(pts)
        live.insert(pts)
        era = inputs.sample_ids(live.live_ids(), n0 // 3, seed=90 + j)
        assert g.erase(dev(era)) == o.erase(era) == live.erase(era)
        gs.append(g)
        os_.append(o)
        qs.append(query_mix(live, m, dim, seed=100 + j))
    out = knn_batch(gs, [dev(q) for q in qs], k)
    torch.cuda.synchronize()
    for j, ((gi, gd), o, q) in enumerate(zip(out, os_, qs)):
        oi, od = oracle_knn(o, q, k)
        assert_rows(gi, gd, oi, od, "forest %d" % j)
    for g in gs:
        g.close()
