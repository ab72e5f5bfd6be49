"""Property checks on an exported static kd-tree (oracle or CUDA library).

A tree export is a dict with the keys produced by OracleForest.tree() and by
the library's tree export: h, nnodes, key, child, box, node_live, leaf_off,
ids, dead.  The checks restate what Sec. IV-A fixes about a static tree:
a complete binary tree laid out in one array, every internal node splitting
its points in half by the median in its dimension, leaves of at most L points,
bounding boxes and live counts of the points below each node.
"""
import numpy as np


def composite_keys(coords_by_id, ids, c):
    ids = np.asarray(ids, dtype=np.int64)
    return (coords_by_id[ids, c].astype(np.int64) << 31) | ids


def check_tree(t, coords_by_id, dim, L):
    h = t["h"]
    nn = t["nnodes"]
    assert nn == (2 << h) - 1
    child = np.asarray(t["child"]).reshape(nn, 2)
    leaf_off = np.asarray(t["leaf_off"], dtype=np.int64)
    ids = np.asarray(t["ids"])
    real_ids = np.where(ids < 0, ids & 0x7FFFFFFF, ids) if ids.dtype == np.int32 else ids
    dead = np.asarray(t["dead"], dtype=bool)
    size = len(ids)
    assert leaf_off[0] == 0 and leaf_off[-1] == size
    assert np.all(np.diff(leaf_off) >= 1), "empty leaf"
    assert np.all(np.diff(leaf_off) <= L), "leaf larger than L"
    seen = np.zeros(nn, dtype=bool)
    box = np.asarray(t["box"]).reshape(nn, 2 * dim)
    live = np.asarray(t["node_live"])
    key = np.asarray(t["key"])

    # iterative DFS carrying (slot, depth, first leaf, leaf count)
    stack = [(0, 0, 0, 1 << h)]
    while stack:
        v, dep, a, nlf = stack.pop()
        assert 0 <= v < nn and not seen[v], "vEB slots must be a permutation"
        seen[v] = True
        lo, hi = leaf_off[a], leaf_off[a + nlf]
        pid = real_ids[lo:hi]
        pts = coords_by_id[pid]
        assert np.array_equal(box[v, :dim], pts.min(axis=0)), "box lo"
        assert np.array_equal(box[v, dim:], pts.max(axis=0)), "box hi"
        assert live[v] == int((~dead[lo:hi]).sum()), "live count"
        if dep == h:
            assert nlf == 1
            assert child[v, 0] == -1 - a, "leaf index"
            continue
        c = dep % dim
        m = hi - lo
        mid = leaf_off[a + nlf // 2]
        assert mid - lo == (m + 1) // 2, "left child must hold ceil(m/2) points"
        kl = composite_keys(coords_by_id, real_ids[lo:mid], c)
        kr = composite_keys(coords_by_id, real_ids[mid:hi], c)
        assert kl.max() == key[v], "split key is the largest key on the left"
        assert kr.min() > key[v], "right keys exceed the split"
        stack.append((int(child[v, 0]), dep + 1, a, nlf // 2))
        stack.append((int(child[v, 1]), dep + 1, a + nlf // 2, nlf // 2))
    assert seen.all()


def leaf_sets(t):
    """Per leaf: sorted ids (erased ones as -1-id), for order-free comparison."""
    ids = np.asarray(t["ids"]).astype(np.int64)
    dead = np.asarray(t["dead"], dtype=bool)
    real = np.where(ids < 0, ids & 0x7FFFFFFF, ids)
    tagged = np.where(dead, -1 - real, real)
    off = np.asarray(t["leaf_off"], dtype=np.int64)
    return [np.sort(tagged[off[i]:off[i + 1]]) for i in range(len(off) - 1)]


def assert_same_tree(a, b, what=""):
    """Bit-exact equality of two exports: shape, keys, children, boxes, live
    counts, leaf ranges and each leaf's id set (within-leaf order is free)."""
    for k in ("h", "nnodes", "size", "live"):
        assert int(a[k]) == int(b[k]), "%s %s: %r != %r" % (what, k, a[k], b[k])
    child_a = np.asarray(a["child"]).reshape(-1, 2)
    child_b = np.asarray(b["child"]).reshape(-1, 2)
    internal = child_a[:, 0] >= 0
    assert np.array_equal(child_a, child_b), what + " children"
    assert np.array_equal(np.asarray(a["key"])[internal], np.asarray(b["key"])[internal]), what + " keys"
    assert np.array_equal(np.asarray(a["box"]).ravel(), np.asarray(b["box"]).ravel()), what + " boxes"
    assert np.array_equal(np.asarray(a["node_live"]).astype(np.int64),
                          np.asarray(b["node_live"]).astype(np.int64)), what + " live"
    assert np.array_equal(np.asarray(a["leaf_off"]).astype(np.int64),
                          np.asarray(b["leaf_off"]).astype(np.int64)), what + " leaf ranges"
    for i, (x, y) in enumerate(zip(leaf_sets(a), leaf_sets(b))):
        assert np.array_equal(x, y), "%s leaf %d ids" % (what, i)


def check_tree_spatial(t, coords_by_id, dim):
    """The spatial-median rule (Sec. V-C): every internal node of depth t splits
    its points in dimension t mod d at v = floor((min + max) / 2) of their
    coordinates (v = 0 for an empty node), key (v << 31) | (2^31 - 1), points
    with coordinate <= v on the left; leaves hold any number of points; boxes
    and live counts are those of the points below (an empty box is
    [INT32_MAX, INT32_MIN])."""
    h = t["h"]
    nn = t["nnodes"]
    assert nn == (2 << h) - 1
    child = np.asarray(t["child"]).reshape(nn, 2)
    leaf_off = np.asarray(t["leaf_off"], dtype=np.int64)
    ids = np.asarray(t["ids"])
    real_ids = np.where(ids < 0, ids & 0x7FFFFFFF, ids) if ids.dtype == np.int32 else ids
    dead = np.asarray(t["dead"], dtype=bool)
    assert leaf_off[0] == 0 and leaf_off[-1] == len(ids)
    assert np.all(np.diff(leaf_off) >= 0)
    box = np.asarray(t["box"]).reshape(nn, 2 * dim)
    live = np.asarray(t["node_live"])
    key = np.asarray(t["key"])
    seen = np.zeros(nn, dtype=bool)
    imax, imin = np.iinfo(np.int32).max, np.iinfo(np.int32).min
    stack = [(0, 0, 0, 1 << h)]
    while stack:
        v, dep, a, nlf = stack.pop()
        assert 0 <= v < nn and not seen[v], "vEB slots must be a permutation"
        seen[v] = True
        lo, hi = leaf_off[a], leaf_off[a + nlf]
        pts = coords_by_id[real_ids[lo:hi]]
        if hi > lo:
            assert np.array_equal(box[v, :dim], pts.min(axis=0)), "box lo"
            assert np.array_equal(box[v, dim:], pts.max(axis=0)), "box hi"
        else:
            assert np.all(box[v, :dim] == imax) and np.all(box[v, dim:] == imin), "empty box"
        assert live[v] == int((~dead[lo:hi]).sum()), "live count"
        if dep == h:
            assert child[v, 0] == -1 - a, "leaf index"
            continue
        c = dep % dim
        sv = (int(pts[:, c].min()) + int(pts[:, c].max())) // 2 if hi > lo else 0
        assert key[v] == (sv << 31) | 0x7FFFFFFF, "spatial split key"
        mid = leaf_off[a + nlf // 2]
        assert np.all(coords_by_id[real_ids[lo:mid], c] <= sv), "left of the split"
        assert np.all(coords_by_id[real_ids[mid:hi], c] > sv), "right of the split"
        stack.append((int(child[v, 0]), dep + 1, a, nlf // 2))
        stack.append((int(child[v, 1]), dep + 1, a + nlf // 2, nlf // 2))
    assert seen.all()
