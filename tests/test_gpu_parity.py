"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Integer work, so the bar is bit-exact: the tree mask, the buffer, every
static tree (node split keys, children, boxes, live counts, leaf ranges and
leaf id sets; within-leaf order is free), the bloom filter words, and every
k-NN row (ids and squared distances) must equal the oracle's after every
batch.  The oracle itself is pinned to the paper in test_oracle_pins.py.
"""
import numpy as np
import pytest
import torch

from oracle.oracle import OracleForest, bruteforce_knn
from paper_2112_06188_gb300 import inputs
from tests.treecheck import assert_same_tree, check_tree

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2112_06188_gb300 import build_lib
    build_lib.build()


def make(dim, L=16, X=1024, **kw):
    from paper_2112_06188_gb300.forest import Forest
    return (Forest(dim, leaf_size=L, buffer_size=X, **kw),
            OracleForest(dim, leaf_size=L, buffer_size=X))


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def assert_same_forest(g, o, coords=None, dim=None, L=None, check_shape=False):
    assert g.tree_mask() == o.tree_mask()
    assert np.array_equal(np.sort(g.buffer_ids()), o.buffer_ids())
    assert g.size() == o.size()
    for lvl in o.tree_levels():
        tg, to = g.tree(lvl), o.tree(lvl)
        assert_same_tree(tg, to, "tree %d" % lvl)
        if to["bloom"] is not None or tg["bloom"] is not None:
            assert tg["bloom"] is not None and to["bloom"] is not None, "bloom built on one side only"
            assert np.array_equal(tg["bloom"], to["bloom"]), "bloom words of tree %d" % lvl
        if check_shape:
            check_tree(tg, coords, dim, L)


def assert_same_knn(g, o, q, k):
    gi, gd = g.knn(to_dev(q), k)
    oi, od = o.knn(q, k)
    gi, gd = gi.cpu().numpy(), gd.cpu().numpy()
    assert np.array_equal(gi, oi), "ids differ in %d rows" % int((gi != oi).any(1).sum())
    assert np.array_equal(gd, od), "d2 differ"
    return gi, gd


SHAPES = [
    # dim, n, L, X
    (2, 1000, 16, 1024),     # buffer only
    (2, 1024, 16, 1024),     # exactly one tree
    (3, 5000, 8, 1024),
    (3, 70000, 16, 1024),    # a 64K tree: global levels + on-chip subtrees
    (5, 40000, 16, 512),
    (7, 30000, 32, 1024),
    (1, 9000, 4, 256),
    (16, 20000, 8, 1024),    # generic dimension path
    (4, 50000, 2, 1024),
    (2, 140000, 8, 4096),
]


@pytest.mark.parametrize("dim,n,L,X", SHAPES)
def test_build_matches_oracle(dim, n, L, X):
    pts = inputs.uniform_points(n, dim, seed=100 + n + dim)
    g, o = make(dim, L, X)
    gi = g.insert(to_dev(pts)).cpu().numpy()
    oi = o.insert(pts)
    assert np.array_equal(gi, oi)
    assert_same_forest(g, o, pts, dim, L, check_shape=True)
    q = np.concatenate([inputs.uniform_points(300, dim, seed=7), pts[:100]])
    for k in (1, 5, 16, 32):
        assert_same_knn(g, o, q, k)


@pytest.mark.parametrize("distinct,n", [(1, 3000), (3, 60000), (40, 90000)])
def test_heavy_ties(distinct, n):
    dim = 2
    pts = inputs.duplicate_heavy_points(n, dim, seed=distinct, distinct=distinct)
    g, o = make(dim, 8, 1024)
    g.insert(to_dev(pts))
    o.insert(pts)
    assert_same_forest(g, o, pts, dim, 8, check_shape=True)
    q = np.concatenate([inputs.uniform_points(100, dim, seed=3), pts[:20]])
    assert_same_knn(g, o, q, 8)
    ids = inputs.sample_ids(np.arange(n), n // 3, seed=5)
    assert g.erase(to_dev(ids)) == o.erase(ids)
    assert_same_forest(g, o)
    assert_same_knn(g, o, q, 8)


def test_clustered_7d():
    dim = 7
    pts = inputs.gaussian_clusters(120000, dim, seed=3, n_clusters=20)
    g, o = make(dim, 16, 1024)
    for a in range(0, len(pts), 40000):
        g.insert(to_dev(pts[a:a + 40000]))
        o.insert(pts[a:a + 40000])
        assert_same_forest(g, o, pts[:a + 40000], dim, 16, check_shape=True)
    q = inputs.gaussian_clusters(2000, dim, seed=4, n_clusters=20)
    assert_same_knn(g, o, q, 5)


def test_small_workload_sequence():
    """The plain small workload (2-D, 65,536 + 8 x 8,192 inserts, 4 x 8,192
    deletes, k = 5 on 4,096 queries after every batch): bit-exact after every
    batch, and the k-NN rows equal brute force."""
    g, o = make(2, 16, 1024)
    live = inputs.LiveSet(2)
    for op, arg in inputs.config_small_sequence(seed=1):
        if op == "insert":
            gi = g.insert(to_dev(arg)).cpu().numpy()
            assert np.array_equal(gi, o.insert(arg))
            live.insert(arg)
        elif op == "erase":
            ne = g.erase(to_dev(arg))
            assert ne == o.erase(arg) == live.erase(arg)
        else:
            gi, gd = assert_same_knn(g, o, arg, 5)
            lp, lid = live.live_points()
            bi, bd = bruteforce_knn(lp, lid, arg[:512], 5)
            assert np.array_equal(gi[:512], bi) and np.array_equal(gd[:512], bd)
            assert_same_forest(g, o, live.coords, 2, 16, check_shape=True)


def test_deep_delete_rebuilds():
    """Erase 70% in ragged batches: trees fall below half and are rebuilt."""
    dim = 3
    g, o = make(dim, 8, 256)
    live = inputs.LiveSet(dim)
    rng = np.random.default_rng(9)
    for n in (70000, 3333, 12345):
        p = rng.integers(0, 1 << 20, size=(n, dim), dtype=np.int32)
        g.insert(to_dev(p))
        o.insert(p)
        live.insert(p)
    q = rng.integers(0, 1 << 20, size=(1000, dim), dtype=np.int32)
    for frac in (0.3, 0.25, 0.2, 0.15):
        ids = inputs.sample_ids(live.live_ids(), int(frac * live.alive.sum()) + 17, seed=int(frac * 100))
        junk = np.array([-1, 10 ** 8, ids[0], ids[1]], np.int32)
        batch = np.concatenate([ids, junk])
        assert g.erase(to_dev(batch)) == o.erase(batch) == live.erase(ids)
        assert_same_forest(g, o, live.coords, dim, 8, check_shape=True)
        for lvl in g.tree_levels():
            assert 2 * g.tree(lvl)["live"] >= 256 << lvl
        gi, _ = assert_same_knn(g, o, q, 10)
        assert not np.isin(gi, np.flatnonzero(~live.alive)).any()
    # and grow again on top of the reinserted trees
    p = rng.integers(0, 1 << 20, size=(20000, dim), dtype=np.int32)
    g.insert(to_dev(p))
    o.insert(p)
    assert_same_forest(g, o)
    assert_same_knn(g, o, q, 10)


def test_multi_tree_batches():
    """Many trees per batch: the 3-D workload scaled down by 64."""
    dim = 3
    g, o = make(dim, 16, 1024)
    rng = np.random.default_rng(2)
    p = rng.integers(0, 1 << 20, size=(156250, dim), dtype=np.int32)
    g.insert(to_dev(p))
    o.insert(p)
    live = inputs.LiveSet(dim)
    live.insert(p)
    assert bin(g.tree_mask()).count("1") >= 3
    for step in range(4):
        p = rng.integers(0, 1 << 20, size=(15625, dim), dtype=np.int32)
        g.insert(to_dev(p))
        o.insert(p)
        live.insert(p)
        assert_same_forest(g, o)
    for step in range(3):
        ids = inputs.sample_ids(live.live_ids(), 15625, seed=step)
        assert g.erase(to_dev(ids)) == o.erase(ids) == live.erase(ids)
        assert_same_forest(g, o)
    q = inputs.queries_from(live.coords[live.alive], 3000, seed=1)
    assert_same_knn(g, o, q, 10)


def test_edge_cases():
    from paper_2112_06188_gb300 import capi
    dim = 2
    g, o = make(dim, 4, 8)
    # empty forest
    q = inputs.uniform_points(5, dim, seed=1)
    gi, gd = g.knn(to_dev(q), 3)
    assert (gi.cpu() == -1).all() and (gd.cpu() == np.iinfo(np.int64).max).all()
    assert g.erase(to_dev(np.array([0, 5, -3], np.int32))) == 0
    # n = 0, m = 0
    g.insert(torch.empty((0, dim), dtype=torch.int32, device="cuda"))
    gi, gd = g.knn(torch.empty((0, dim), dtype=torch.int32, device="cuda"), 4)
    assert gi.shape == (0, 4)
    # out-of-grid coordinates: EINVAL, forest unchanged
    with pytest.raises(capi.BdlError) as e:
        g.insert(to_dev(np.array([[0, 1 << 20]], np.int32)))
    assert e.value.status == capi.BDL_EINVAL
    with pytest.raises(capi.BdlError):
        g.insert(to_dev(np.array([[-1, 0]], np.int32)))
    assert g.size() == 0 and g.tree_mask() == 0
    # bad k
    with pytest.raises(capi.BdlError):
        g.knn(to_dev(q), 0)
    with pytest.raises(capi.BdlError):
        g.knn(to_dev(q), 33)
    # fewer live points than k; ids restart where they should after the EINVAL
    p = np.array([[1, 1], [3, 3], [5, 5]], np.int32)
    assert list(g.insert(to_dev(p)).cpu().numpy()) == [0, 1, 2]
    o.insert(p)
    gi, gd = assert_same_knn(g, o, np.array([[0, 0]], np.int32), 5)
    assert list(gi[0]) == [0, 1, 2, -1, -1]
    # grow through several trees, erase everything, reuse
    p2 = inputs.uniform_points(100, dim, seed=2)
    g.insert(to_dev(p2))
    o.insert(p2)
    assert_same_forest(g, o)
    all_ids = np.arange(103, dtype=np.int32)
    assert g.erase(to_dev(all_ids)) == o.erase(all_ids) == 103
    assert g.size() == 0 and g.tree_mask() == 0
    assert_same_knn(g, o, q, 2)
    g.insert(to_dev(p2[:9]))
    o.insert(p2[:9])
    assert_same_forest(g, o)
    assert_same_knn(g, o, q, 32)


def test_erase_batches_that_erase_nothing():
    """A batch with no live id (never inserted, negative, already erased,
    repeated) changes nothing, not even the lazy bloom filters (Sec. V-A):
    they are built by the first erase that erases something."""
    dim = 3
    g, o = make(dim, 16, 64)
    p = inputs.uniform_points(5000, dim, seed=21)
    g.insert(to_dev(p))
    o.insert(p)
    dead = np.array([50000, 70000, -1, 123456, 50000], np.int32)   # never inserted
    assert g.erase(to_dev(dead)) == o.erase(dead) == 0
    assert_same_forest(g, o)
    assert all(g.tree(lvl)["bloom"] is None for lvl in o.tree_levels())
    ids = np.arange(0, 5000, 7, dtype=np.int32)
    assert g.erase(to_dev(ids)) == o.erase(ids) == len(ids)
    assert_same_forest(g, o)
    assert all(g.tree(lvl)["bloom"] is not None for lvl in o.tree_levels())
    again = np.concatenate([ids[:50], ids[:50], dead])
    assert g.erase(to_dev(again)) == o.erase(again) == 0
    p2 = inputs.uniform_points(3000, dim, seed=23)   # new trees: blooms unbuilt again
    g.insert(to_dev(p2))
    o.insert(p2)
    assert g.erase(to_dev(again)) == o.erase(again) == 0
    assert_same_forest(g, o)
    assert_same_knn(g, o, inputs.uniform_points(300, dim, seed=22), 10)


@pytest.mark.parametrize("dim", [2, 3, 4])
def test_knn_counting_instance(dim):
    """With visit counting on, k-NN runs its counting instance (a plain walk of
    the binary nodes instead of the packed records): the rows are the same as
    the timed instance's and the oracle's, and every query is counted."""
    g, o = make(dim, 16, 256)
    n = 40000
    p = inputs.uniform_points(n, dim, seed=31)
    g.insert(to_dev(p))
    o.insert(p)
    ids = inputs.sample_ids(np.arange(n, dtype=np.int32), 9000, seed=32)
    assert g.erase(to_dev(ids)) == o.erase(ids)
    q = inputs.uniform_points(5000, dim, seed=33)
    gi, gd = assert_same_knn(g, o, q, 7)
    g.knn_stats(True)
    si, sd = g.knn(to_dev(q), 7)
    nodes, points, nq = g.knn_stats()
    g.knn_stats(False)
    assert np.array_equal(si.cpu().numpy(), gi) and np.array_equal(sd.cpu().numpy(), gd)
    assert nq == len(q) and nodes >= len(q) and points >= 7 * len(q)


@pytest.mark.parametrize("dim", [2, 3])
def test_small_erase_batches(dim):
    """Erase batches under 1/128 of the forest keep the packed k-NN records'
    live counts on their descent paths (debug runs compare every record with
    its nodes after each erase); results stay the oracle's."""
    g, o = make(dim, 8, 128)
    n = 60000
    p = inputs.uniform_points(n, dim, seed=41)
    g.insert(to_dev(p))
    o.insert(p)
    live = np.arange(n, dtype=np.int32)
    q = inputs.uniform_points(2000, dim, seed=42)
    for step in range(12):
        ids = inputs.sample_ids(live, 60 + 17 * step, seed=43 + step)
        ids = np.concatenate([ids, ids[:5], np.array([n + 7, -2], np.int32)])   # repeats, dead ids
        assert g.erase(to_dev(ids)) == o.erase(ids)
        live = np.setdiff1d(live, ids)
        if step % 4 == 3:
            assert_same_forest(g, o)
            assert_same_knn(g, o, q, 9)
    ins = inputs.uniform_points(3000, dim, seed=44)     # new trees, then more small erases
    g.insert(to_dev(ins))
    o.insert(ins)
    ids = inputs.sample_ids(np.arange(n + 3000, dtype=np.int32), 300, seed=45)
    assert g.erase(to_dev(ids)) == o.erase(ids)
    assert_same_forest(g, o)
    assert_same_knn(g, o, q, 9)


def test_host_buffers_end_to_end():
    """The public API with host (numpy) arrays copies in and out itself."""
    dim = 3
    pts = inputs.uniform_points(30000, dim, seed=5)
    g, o = make(dim)
    gi = g.insert(pts)
    assert isinstance(gi, torch.Tensor) and not gi.is_cuda
    o.insert(pts)
    q = inputs.uniform_points(500, dim, seed=6)
    hi, hd = g.knn(q, 7)
    oi, od = o.knn(q, 7)
    assert np.array_equal(hi.numpy(), oi) and np.array_equal(hd.numpy(), od)
    assert g.erase(np.arange(0, 30000, 3, dtype=np.int32)) == o.erase(np.arange(0, 30000, 3, dtype=np.int32))
    assert_same_forest(g, o)


def test_streams_and_budget():
    from paper_2112_06188_gb300 import capi
    from paper_2112_06188_gb300.forest import Forest
    s = torch.cuda.Stream()
    dim = 2
    pts = inputs.uniform_points(50000, dim, seed=8)
    g = Forest(dim, stream=s)
    o = OracleForest(dim)
    with torch.cuda.stream(s):
        d = to_dev(pts)
    g.insert(d)
    o.insert(pts)
    q = inputs.uniform_points(1000, dim, seed=9)
    hi, hd = g.knn(q, 4)
    oi, od = o.knn(q, 4)
    assert np.array_equal(hi.numpy(), oi)
    # a tight budget refuses the build and leaves the forest as it was
    small = Forest(dim, hbm_budget_bytes=1 << 20)
    small.insert(pts[:1000])
    with pytest.raises(capi.BdlError) as e:
        small.insert(to_dev(pts))
    assert e.value.status == capi.BDL_ENOMEM
    assert small.size() == 1000
    o2 = OracleForest(dim)
    o2.insert(pts[:1000])
    assert_same_knn(small, o2, q, 3)
