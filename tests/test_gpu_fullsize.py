"""Parity at full size, in the configuration bench.py times.

At 10M points the oracle cannot replay the whole sequence in test time, so
these tests check what holds at any size:
  * 1,000 sampled k-NN rows per call equal brute force over the live set
    (exact, bit for bit), in the launch configuration the benchmark times
    (1M queries, spatial order),
  * no erased id ever appears in a result, every row is sorted by (d2, id),
  * the live count matches, and every static tree holds at least half of its
    capacity X * 2^i after every erase (Alg. 4), insert-only trees exactly fill
    theirs (Sec. III-D),
  * every static tree of at most 2M points is a valid median-split kd-tree in
    vEB layout (Alg. 1: node keys, children, boxes, live counts, leaf ranges)
    after every phase.
"""
import numpy as np
import pytest
import torch

from paper_2112_06188_gb300 import inputs
from oracle.threads import bruteforce_knn_threads
from tests.treecheck import check_tree

pytestmark = pytest.mark.gpu

X = 1024


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2112_06188_gb300 import build_lib
    build_lib.build()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def check_invariants(f, live, insert_only):
    assert f.size() == int(live.alive.sum())
    total = len(f.buffer_ids())
    for lvl in f.tree_levels():
        t = f.tree(lvl)
        total += t["live"]
        if insert_only:
            assert t["size"] == X << lvl and t["live"] == t["size"]
        else:
            assert 2 * t["live"] >= X << lvl
    assert total == f.size()


def check_trees(f, live, dim, L, max_size=2_000_000):
    """check_tree on every static tree of at most max_size points."""
    done = 0
    for lvl in f.tree_levels():
        t = f.tree(lvl)
        if t["size"] <= max_size:
            check_tree(t, live.coords, dim, L)
            done += 1
    assert done > 0


def check_knn(f, live, q, k, sample, seed):
    gi, gd = f.knn(dev(q), k)
    gi, gd = gi.cpu().numpy(), gd.cpu().numpy()
    # rows sorted by (d2, id), no erased ids
    assert np.all((gd[:, 1:] > gd[:, :-1]) | ((gd[:, 1:] == gd[:, :-1]) & (gi[:, 1:] > gi[:, :-1])))
    assert live.alive[gi.ravel()].all()
    rows = np.random.default_rng(seed).choice(len(q), size=sample, replace=False)
    lp, lid = live.live_points()
    bi, bd = bruteforce_knn_threads(lp, lid, q[rows], k)
    assert np.array_equal(gi[rows], bi)
    assert np.array_equal(gd[rows], bd)


def test_uniform_3d_10M_sequence():
    """10M uniform 3-D points, 1M inserts and 1M deletes of live ids, k = 10 for
    1M live-set queries after each phase (leaf 16, X = 1024)."""
    from paper_2112_06188_gb300.forest import Forest
    dim, k, n0, b, m = 3, 10, 10_000_000, 1_000_000, 1_000_000
    rng = np.random.default_rng(2)
    live = inputs.LiveSet(dim)
    f = Forest(dim, leaf_size=16, buffer_size=X)
    p = rng.integers(0, 1 << 20, size=(n0, dim), dtype=np.int32)
    ids = f.insert(dev(p)).cpu().numpy()
    assert np.array_equal(ids, live.insert(p))
    check_invariants(f, live, insert_only=True)
    check_trees(f, live, dim, 16)
    check_knn(f, live, inputs.queries_from(p, m, seed=3), k, 1000, seed=4)
    for step in range(3):
        p = rng.integers(0, 1 << 20, size=(b, dim), dtype=np.int32)
        f.insert(dev(p))
        live.insert(p)
        check_invariants(f, live, insert_only=True)
    check_trees(f, live, dim, 16)
    check_knn(f, live, inputs.queries_from(live.coords[live.alive], m, seed=5), k, 1000, seed=6)
    for step in range(3):
        era = inputs.sample_ids(live.live_ids(), b, seed=10 + step)
        assert f.erase(dev(era)) == live.erase(era) == b
        check_invariants(f, live, insert_only=False)
    check_trees(f, live, dim, 16)
    check_knn(f, live, inputs.queries_from(live.coords[live.alive], m, seed=7), k, 1000, seed=8)
    f.close()


def test_clustered_7d_10M_mixed_batches():
    """10M points from 100 Gaussian clusters in 7-D; insert and delete batches of
    10%, 1% and 0.1% of n; k = 5 for 1M queries from the same mixture."""
    from paper_2112_06188_gb300.forest import Forest
    dim, k, n0, m = 7, 5, 10_000_000, 1_000_000
    pts = inputs.gaussian_clusters(n0 + n0 // 10 + n0 // 100 + n0 // 1000, dim, seed=3)
    live = inputs.LiveSet(dim)
    f = Forest(dim, leaf_size=16, buffer_size=X)
    f.insert(dev(pts[:n0]))
    live.insert(pts[:n0])
    q = inputs.gaussian_clusters(m, dim, seed=4)
    check_knn(f, live, q, k, 1000, seed=5)
    a = n0
    for frac in (10, 100, 1000):
        nb = n0 // frac
        f.insert(dev(pts[a:a + nb]))
        live.insert(pts[a:a + nb])
        a += nb
        era = inputs.sample_ids(live.live_ids(), nb, seed=frac)
        assert f.erase(dev(era)) == live.erase(era)
        check_invariants(f, live, insert_only=False)
    check_trees(f, live, dim, 16)
    check_knn(f, live, q, k, 1000, seed=6)
    f.close()
