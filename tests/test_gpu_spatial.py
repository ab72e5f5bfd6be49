"""Parity of the spatial-median build (Sec. V-C, reading G12) with the oracle.

Same bar as the object-median parity: after every batch the tree masks,
buffers, every tree's node keys, children, boxes, live counts, leaf ranges and
leaf id sets (order inside a leaf is free), the bloom words and every k-NN
row are bit-exact; every GPU tree also satisfies the spatial split invariant
directly (tests/treecheck.py), and sampled k-NN rows equal brute force.
"""
import numpy as np
import pytest
import torch

from oracle.oracle import OracleForest, bruteforce_knn
from paper_2112_06188_gb300 import inputs
from tests.treecheck import check_tree_spatial
from tests.test_gpu_parity import assert_same_forest, assert_same_knn, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2112_06188_gb300 import build_lib
    build_lib.build()


def make(dim, L=16, X=1024):
    from paper_2112_06188_gb300.forest import Forest
    return (Forest(dim, leaf_size=L, buffer_size=X, split="spatial"),
            OracleForest(dim, leaf_size=L, buffer_size=X, split="spatial"))


def same(g, o, coords, dim):
    assert_same_forest(g, o)
    for lvl in g.tree_levels():
        check_tree_spatial(g.tree(lvl), coords, dim)


def line_points(n, dim, seed):
    p = np.zeros((n, dim), np.int32)
    p[:, 0] = np.random.default_rng(seed).integers(0, 1 << 20, n)
    return p


SHAPES = [
    # dim, n, L, X, generator
    (2, 1000, 16, 1024, "uniform"),      # buffer only
    (2, 1024, 16, 1024, "uniform"),      # one tree
    (3, 70000, 16, 1024, "uniform"),
    (3, 60000, 8, 1024, "clusters"),
    (5, 40000, 16, 512, "uniform"),
    (7, 30000, 32, 1024, "clusters"),
    (1, 9000, 4, 256, "uniform"),
    (16, 20000, 8, 1024, "uniform"),
    (2, 50000, 2, 1024, "duplicates"),   # many empty subtrees, some huge leaves
    (3, 40000, 8, 512, "line"),          # every other split is degenerate
]


def points(gen, n, dim, seed):
    if gen == "uniform":
        return inputs.uniform_points(n, dim, seed)
    if gen == "clusters":
        return inputs.gaussian_clusters(n, dim, seed, n_clusters=7)
    if gen == "duplicates":
        return inputs.duplicate_heavy_points(n, dim, seed, distinct=5)
    return line_points(n, dim, seed)


@pytest.mark.parametrize("dim,n,L,X,gen", SHAPES)
def test_spatial_build_matches_oracle(dim, n, L, X, gen):
    pts = points(gen, n, dim, seed=n + dim)
    g, o = make(dim, L, X)
    assert np.array_equal(g.insert(to_dev(pts)).cpu().numpy(), o.insert(pts))
    same(g, o, pts, dim)
    q = np.concatenate([inputs.uniform_points(300, dim, seed=7), pts[:100]])
    for k in (1, 8, 32):
        assert_same_knn(g, o, q, k)
    g.close()


def test_spatial_sequence_with_rebuilds():
    """Inserts, erases deep enough to empty and rebuild trees, more inserts;
    bit-exact after every batch and the k-NN rows equal brute force."""
    dim = 3
    g, o = make(dim, 8, 256)
    live = inputs.LiveSet(dim)
    rng = np.random.default_rng(4)
    for n in (50000, 4321, 20000):
        p = inputs.gaussian_clusters(n, dim, seed=n, n_clusters=5)
        g.insert(to_dev(p))
        o.insert(p)
        live.insert(p)
        same(g, o, live.coords, dim)
    q = rng.integers(0, 1 << 20, size=(800, dim), dtype=np.int32)
    for frac in (0.35, 0.3, 0.25):
        ids = inputs.sample_ids(live.live_ids(), int(frac * live.alive.sum()), seed=int(frac * 100))
        assert g.erase(to_dev(ids)) == o.erase(ids) == live.erase(ids)
        same(g, o, live.coords, dim)
        gi, gd = assert_same_knn(g, o, q, 6)
        lp, lid = live.live_points()
        bi, bd = bruteforce_knn(lp, lid, q[:200], 6)
        assert np.array_equal(gi[:200], bi) and np.array_equal(gd[:200], bd)
    p = rng.integers(0, 1 << 20, size=(30000, dim), dtype=np.int32)
    g.insert(to_dev(p))
    o.insert(p)
    live.insert(p)
    same(g, o, live.coords, dim)
    assert_same_knn(g, o, q, 6)
    g.close()


def test_spatial_and_object_answer_alike():
    """The splitting rule changes the trees, not the answers."""
    from paper_2112_06188_gb300.forest import Forest
    dim = 3
    a = Forest(dim, leaf_size=16, split="spatial")
    b = Forest(dim, leaf_size=16)
    p = inputs.gaussian_clusters(120000, dim, seed=1, n_clusters=9)
    a.insert(to_dev(p))
    b.insert(to_dev(p))
    e = inputs.sample_ids(np.arange(len(p)), 30000, seed=2)
    assert a.erase(to_dev(e)) == b.erase(to_dev(e))
    q = to_dev(inputs.gaussian_clusters(40000, dim, seed=3, n_clusters=9))
    ai, ad = a.knn(q, 10)
    bi, bd = b.knn(q, 10)
    assert torch.equal(ai, bi) and torch.equal(ad, bd)
    a.close()
    b.close()


def test_spatial_in_mixed_batches():
    """Spatial and object forests in one batched call build in separate classes;
    each forest gets its single-call result."""
    from paper_2112_06188_gb300.forest import Forest, erase_batch, insert_batch, knn_batch
    dims = [2, 3, 3, 2, 5, 3]
    rules = ["spatial", "object", "spatial", "object", "spatial", "spatial"]
    A = [Forest(d, split=r) for d, r in zip(dims, rules)]
    B = [Forest(d, split=r) for d, r in zip(dims, rules)]
    pts = [inputs.gaussian_clusters(5000 + 3000 * i, d, seed=i, n_clusters=4) for i, d in enumerate(dims)]
    insert_batch(A, [to_dev(p) for p in pts])
    for f, p in zip(B, pts):
        f.insert(to_dev(p))
    ids = [inputs.sample_ids(np.arange(len(p)), len(p) // 2 + 7, seed=i) for i, p in enumerate(pts)]
    assert erase_batch(A, [to_dev(e) for e in ids]) == [f.erase(to_dev(e)) for f, e in zip(B, ids)]
    for f, g in zip(A, B):
        assert_same_forest(f, g)
    qs = [to_dev(inputs.uniform_points(700, d, seed=9)) for d in dims]
    out = knn_batch(A, qs, 7)
    for (ai, ad), f, q in zip(out, B, qs):
        bi, bd = f.knn(q, 7)
        assert torch.equal(ai, bi) and torch.equal(ad, bd)
    for f in A + B:
        f.close()
