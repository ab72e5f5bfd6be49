"""Pins of the CPU oracle against what the paper and the mathematics fix.

* Sec. IV-A1 / Fig. 3: the vEB worked example (bottom subtrees at 3, 6, 9, 12).
* Sec. IV-B1 / Fig. 4: the insert worked example (F = 1, 2, 3, 4).
* Sec. III-D: insert-only forests hold the binary counter of floor(n/X).
* Sec. IV-A1: every internal node halves its points at the median (tree check).
* Alg. 4: no static tree below half capacity after an erase; erased ids never
  come back; ids that are not live are ignored.
* The exact k-NN result by definition (brute force), including ties, k > n
  and queries on top of points.
* Sec. V-A: a bloom filter has no false negatives.
* SplitMix64's published first output for seed 0.
"""
import os

import numpy as np
import pytest

from oracle.oracle import OracleForest, bruteforce_knn, splitmix64
from paper_2112_06188_gb300 import inputs
from tests.treecheck import check_tree

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def read_golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


def hyperceil_half(l):
    lb = 1
    while 2 * lb < l:
        lb *= 2
    return lb


def veb_slot(l, t, i):
    """Closed form of the vEB position of node (depth t, index i) in a tree
    of l levels (independent of the oracle's recursive construction)."""
    if l == 1:
        return 0
    lb = hyperceil_half(l)
    lt = l - lb
    if t < lt:
        return veb_slot(lt, t, i)
    tt = t - lt
    j = i >> tt
    return (2 ** lt - 1) + j * (2 ** lb - 1) + veb_slot(lb, tt, i & ((1 << tt) - 1))


def test_veb_worked_example():
    pts = np.array([[1, 1], [3, 3], [5, 5], [7, 7], [2, 6], [6, 2], [4, 0], [0, 4]], np.int32)
    f = OracleForest(2, leaf_size=1, buffer_size=8)
    f.insert(pts)
    assert f.tree_levels() == [0]
    t = f.tree(0)
    assert t["h"] == 3 and t["nnodes"] == 15
    for slot, depth, idx in read_golden("veb_worked_example.txt"):
        assert t["depth"][int(slot)] == int(depth)
        assert t["bfs"][int(slot)] == int(idx)
    # every bottom subtree is laid out contiguously: root, then its 2 leaves
    for r in (3, 6, 9, 12):
        assert list(t["depth"][r:r + 3]) == [2, 3, 3]


@pytest.mark.parametrize("n", [2 ** 9, 5000, 20000])
def test_veb_slots_match_closed_form(n):
    pts = inputs.uniform_points(n, 3, seed=n)
    f = OracleForest(3, leaf_size=4, buffer_size=n)
    f.insert(pts)
    t = f.tree(0)
    l = t["h"] + 1
    for v in range(t["nnodes"]):
        assert veb_slot(l, int(t["depth"][v]), int(t["bfs"][v])) == v


@pytest.mark.parametrize("X", [3, 4, 16])
def test_insert_worked_example(X):
    f = OracleForest(2, leaf_size=2, buffer_size=X)
    rng = np.random.default_rng(7)
    for step, F, nbuf in read_golden("insert_fig4.txt"):
        n = X + int(step[1:]) if step.startswith("X") else int(step)
        f.insert(rng.integers(0, 1 << 20, size=(n, 2), dtype=np.int32))
        assert f.tree_mask() == int(F)
        assert len(f.buffer_ids()) == int(nbuf)


def test_binary_counter_and_tree_shape():
    X, L, dim = 64, 8, 3
    f = OracleForest(dim, leaf_size=L, buffer_size=X)
    rng = np.random.default_rng(3)
    coords = np.empty((0, dim), np.int32)
    n = 0
    for b in [1, 63, 64, 65, 1000, 7, 4096, 333]:
        p = rng.integers(0, 1 << 20, size=(b, dim), dtype=np.int32)
        coords = np.concatenate([coords, p])
        f.insert(p)
        n += b
        assert f.tree_mask() == n // X
        assert len(f.buffer_ids()) == n % X
        for lvl in f.tree_levels():
            t = f.tree(lvl)
            assert t["size"] == X << lvl
            check_tree(t, coords, dim, L)


def test_tree_shape_with_duplicates():
    dim, L = 2, 4
    pts = inputs.duplicate_heavy_points(3000, dim, seed=5, distinct=3)
    f = OracleForest(dim, leaf_size=L, buffer_size=1000)
    f.insert(pts)
    for lvl in f.tree_levels():
        check_tree(f.tree(lvl), pts, dim, L)


@pytest.mark.parametrize("dim,k,gen", [(2, 5, "uniform"), (3, 10, "uniform"), (5, 1, "clusters"),
                                       (7, 8, "clusters"), (2, 6, "dups"), (1, 3, "uniform")])
def test_knn_matches_bruteforce(dim, k, gen):
    n = 3000
    if gen == "uniform":
        pts = inputs.uniform_points(n, dim, seed=11)
    elif gen == "clusters":
        pts = inputs.gaussian_clusters(n, dim, seed=12, n_clusters=5)
    else:
        pts = inputs.duplicate_heavy_points(n, dim, seed=13, distinct=5)
    f = OracleForest(dim, leaf_size=4, buffer_size=128)
    live = inputs.LiveSet(dim)
    for a in range(0, n, 700):
        f.insert(pts[a:a + 700])
        live.insert(pts[a:a + 700])
    q = np.concatenate([inputs.uniform_points(200, dim, seed=14), pts[:50]])
    got = f.knn(q, k)
    lp, lid = live.live_points()
    want = bruteforce_knn(lp, lid, q, k)
    assert np.array_equal(got[0], want[0])
    assert np.array_equal(got[1], want[1])
    # a query on top of a live point finds it at distance 0
    assert np.all(got[1][200:, 0] == 0)


def test_knn_more_neighbours_than_points():
    f = OracleForest(2, leaf_size=2, buffer_size=4)
    pts = np.array([[1, 1], [3, 3], [5, 5], [7, 7], [9, 9], [11, 11]], np.int32)
    f.insert(pts)
    ids, d2 = f.knn(np.array([[0, 0]], np.int32), 8)
    assert list(ids[0]) == [0, 1, 2, 3, 4, 5, -1, -1]
    assert list(d2[0][:6]) == [2, 18, 50, 98, 162, 242]
    assert d2[0][6] == np.iinfo(np.int64).max


def test_bruteforce_small_by_hand():
    pts = np.array([[0, 0], [2, 0], [0, 2], [1, 1]], np.int32)
    ids = np.array([10, 11, 12, 13], np.int32)
    got_ids, got_d2 = bruteforce_knn(pts, ids, np.array([[1, 0]], np.int32), 3)
    # distances: 1, 1, 5, 1 -> ties broken by id
    assert list(got_ids[0]) == [10, 11, 13]
    assert list(got_d2[0]) == [1, 1, 1]


def test_erase_semantics_and_half_invariant():
    X, L, dim = 32, 4, 2
    f = OracleForest(dim, leaf_size=L, buffer_size=X)
    live = inputs.LiveSet(dim)
    rng = np.random.default_rng(21)
    for b in [500, 300, 77]:
        p = rng.integers(0, 1 << 20, size=(b, dim), dtype=np.int32)
        f.insert(p)
        live.insert(p)
    for step in range(8):
        ids = rng.choice(live.live_ids(), size=min(90, len(live.live_ids())), replace=False)
        junk = np.array([-5, 10 ** 6, ids[0], ids[0]], np.int32)   # not live / repeated
        batch = np.concatenate([ids.astype(np.int32), junk])
        n = f.erase(batch)
        assert n == live.erase(ids)
        assert f.size() == int(live.alive.sum())
        for lvl in f.tree_levels():
            t = f.tree(lvl)
            assert 2 * t["live"] >= X << lvl, "tree below half after Erase_L"
            check_tree(t, live.coords, dim, L)
        q = rng.integers(0, 1 << 20, size=(64, dim), dtype=np.int32)
        got = f.knn(q, 7)
        lp, lid = live.live_points()
        want = bruteforce_knn(lp, lid, q, 7)
        assert np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1])
        assert not np.isin(got[0], np.flatnonzero(~live.alive)).any()
    assert f.erase(np.array([], np.int32)) == 0


def test_erase_everything_then_reinsert():
    f = OracleForest(3, leaf_size=4, buffer_size=16)
    pts = inputs.uniform_points(1000, 3, seed=4)
    ids = f.insert(pts)
    assert f.erase(ids) == 1000
    assert f.size() == 0 and f.tree_mask() == 0 and len(f.buffer_ids()) == 0
    out_ids, out_d2 = f.knn(pts[:3], 2)
    assert np.all(out_ids == -1)
    ids2 = f.insert(pts[:40])
    assert ids2[0] == 1000 and f.size() == 40


def test_insert_rejects_out_of_grid():
    f = OracleForest(2)
    with pytest.raises(ValueError):
        f.insert(np.array([[0, 1 << 20]], np.int32))
    with pytest.raises(ValueError):
        f.insert(np.array([[-1, 0]], np.int32))
    assert f.size() == 0


def test_bloom_no_false_negatives_and_rate():
    X, dim = 256, 2
    f = OracleForest(dim, leaf_size=8, buffer_size=X, bloom_bits_per_key=16)
    pts = inputs.uniform_points(X * 7, dim, seed=8)
    f.insert(pts)
    f.erase(np.array([0], np.int32))          # first erase builds every filter
    members = 0
    false_pos = 0
    probes = 0
    for lvl in f.tree_levels():
        t = f.tree(lvl)
        assert t["bloom"] is not None
        for pid, dead in zip(t["ids"], t["dead"]):
            if not dead:
                assert f.bloom_maybe(lvl, pid) == 1
                members += 1
        others = np.setdiff1d(np.arange(X * 7), t["ids"])
        for pid in others:
            false_pos += f.bloom_maybe(lvl, pid)
            probes += 1
    assert members == X * 7 - 1
    assert false_pos / probes < 0.01


def test_splitmix64_published_vector():
    # first output of SplitMix64 seeded with 0 (Steele, Lea & Flood 2014)
    assert splitmix64(0) == 0xE220A8397B1DCDAF


def test_small_workload_sequence_against_bruteforce():
    """The plain small workload, scaled down 16x, replayed through the oracle."""
    f = OracleForest(2, leaf_size=16, buffer_size=1024)
    live = inputs.LiveSet(2)
    for op, arg in inputs.config_small_sequence(seed=1, n0=4096, ins=512, dele=512, m=256):
        if op == "insert":
            f.insert(arg)
            live.insert(arg)
        elif op == "erase":
            assert f.erase(arg) == live.erase(arg)
        else:
            got = f.knn(arg, 5)
            lp, lid = live.live_points()
            want = bruteforce_knn(lp, lid, arg, 5)
            assert np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1])


def test_below_half_is_strict():
    """Alg. 4 rebuilds trees that drop *below* half capacity: exactly half stays."""
    X = 4
    f = OracleForest(2, leaf_size=2, buffer_size=X)
    ids = f.insert(inputs.uniform_points(2 * X, 2, seed=9))     # one tree of capacity 2X
    assert f.tree_mask() == 2
    assert f.erase(ids[:X]) == X                                  # live == cap/2
    assert f.tree_mask() == 2 and f.tree(1)["live"] == X
    assert f.erase(ids[X:X + 1]) == 1                             # live < cap/2
    assert f.tree_mask() == 0 and sorted(f.buffer_ids()) == list(ids[X + 1:])
    # the X-1 survivors went to the buffer; one more point makes tree 0
    f.insert(inputs.uniform_points(1, 2, seed=10))
    assert f.tree_mask() == 1 and len(f.buffer_ids()) == 0


# --- the spatial-median rule (Sec. V-C) ------------------------------------

def test_spatial_worked_example():
    from tests.treecheck import check_tree_spatial
    rows = read_golden("spatial_fig1.txt")
    pts = np.array([[int(r[1]), int(r[2])] for r in rows if r[0] == "point"], np.int32)
    (_, dim0, split, left, right), = [r for r in rows if r[0] == "root"]
    f = OracleForest(2, leaf_size=1, buffer_size=2, split="spatial")
    f.insert(pts)
    t = f.tree(0)
    assert t["h"] == 1
    assert int(t["key"][0]) >> 31 == int(split) and int(dim0) == 0 % 2
    off = t["leaf_off"]
    assert list(t["ids"][off[0]:off[1]]) == [int(left)]
    assert list(t["ids"][off[1]:off[2]]) == [int(right)]
    check_tree_spatial(t, pts, 2)


@pytest.mark.parametrize("gen", ["uniform", "clusters", "duplicates", "line"])
def test_spatial_tree_shape(gen):
    from tests.treecheck import check_tree_spatial
    dim = 3
    if gen == "uniform":
        pts = inputs.uniform_points(9000, dim, seed=1)
    elif gen == "clusters":
        pts = inputs.gaussian_clusters(9000, dim, seed=2, n_clusters=5)
    elif gen == "duplicates":
        pts = inputs.duplicate_heavy_points(9000, dim, seed=3, distinct=4)
    else:                      # all points on one axis: every other level splits nothing
        pts = np.zeros((9000, dim), np.int32)
        pts[:, 0] = np.random.default_rng(4).integers(0, 1 << 20, 9000)
    f = OracleForest(dim, leaf_size=8, buffer_size=1024, split="spatial")
    f.insert(pts)
    for lvl in f.tree_levels():
        check_tree_spatial(f.tree(lvl), pts, dim)
    ids = inputs.sample_ids(np.arange(len(pts)), 4000, seed=5)
    f.erase(ids)
    for lvl in f.tree_levels():
        check_tree_spatial(f.tree(lvl), pts, dim)


@pytest.mark.parametrize("dim,k", [(2, 5), (3, 10), (5, 1)])
def test_spatial_knn_matches_bruteforce(dim, k):
    live = inputs.LiveSet(dim)
    f = OracleForest(dim, leaf_size=8, buffer_size=256, split="spatial")
    g = OracleForest(dim, leaf_size=8, buffer_size=256)
    rng = np.random.default_rng(dim)
    for step in range(4):
        p = inputs.gaussian_clusters(3000, dim, seed=10 + step, n_clusters=6)
        live.insert(p)
        f.insert(p)
        g.insert(p)
        e = inputs.sample_ids(live.live_ids(), 1200, seed=20 + step)
        assert f.erase(e) == live.erase(e) == g.erase(e)
        q = np.concatenate([rng.integers(0, 1 << 20, (150, dim), dtype=np.int32), p[:50]])
        lp, lid = live.live_points()
        bi, bd = bruteforce_knn(lp, lid, q, k)
        fi, fd = f.knn(q, k)
        gi, gd = g.knn(q, k)
        assert np.array_equal(fi, bi) and np.array_equal(fd, bd)
        assert np.array_equal(gi, fi) and np.array_equal(gd, fd)
