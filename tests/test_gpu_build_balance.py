"""Builds whose on-chip subtrees are rebalanced by extra global levels.

A build gives the trees that have fewer global median levels than its deepest
tree extra ones when an estimated schedule of the subtree CTAs finishes
sooner; the trees (Alg. 1's median splits, vEB layout) must not change.  On a
whole GPU that choice arises only for builds of millions of points, so these
tests schedule on a few slots (BDL_BUILD_SLOTS), chosen so that the builds of
tens of thousands of points here take extra levels, and compare every tree
with the oracle's, bit for bit, in 2, 3, 5 and 7 dimensions, through single
and batched inserts and the rebuilds of an erase (Alg. 3, Alg. 4)."""
import numpy as np
import pytest
import torch

from oracle.oracle import OracleForest
from paper_2112_06188_gb300 import inputs
from tests.treecheck import assert_same_tree

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2112_06188_gb300 import build_lib
    build_lib.build()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def same_forest(g, o, what):
    assert g.tree_mask() == o.tree_mask(), what
    assert g.size() == o.size(), what
    for lvl in o.tree_levels():
        assert_same_tree(g.tree(lvl), o.tree(lvl), "%s, tree %d" % (what, lvl))


# slots for which the schedule model deepens the initial build's smaller trees
@pytest.mark.parametrize("dim,n,slots", [(3, 130_000, 7), (2, 200_000, 7), (5, 100_000, 7), (7, 70_000, 8)])
def test_single_forest_builds(dim, n, slots, monkeypatch):
    from paper_2112_06188_gb300.forest import Forest
    monkeypatch.setenv("BDL_BUILD_SLOTS", str(slots))
    g, o = Forest(dim), OracleForest(dim)
    pts = inputs.uniform_points(n, dim, seed=700 + dim)
    g.insert(dev(pts))
    o.insert(pts)
    same_forest(g, o, "initial build")
    more = inputs.uniform_points(n // 2 + 333, dim, seed=710 + dim)   # a carry into bigger trees
    g.insert(dev(more))
    o.insert(more)
    same_forest(g, o, "after an insert")
    era = inputs.sample_ids(np.arange(n + n // 2 + 333), int(0.6 * g.size()), seed=720 + dim)
    assert g.erase(dev(era)) == o.erase(era)                          # below-half rebuilds
    same_forest(g, o, "after an erase")
    g.close()


def test_batched_builds_mixed_dims(monkeypatch):
    from paper_2112_06188_gb300.forest import Forest, insert_batch
    monkeypatch.setenv("BDL_BUILD_SLOTS", "10")   # deepens each dimension's build
    specs = [(3, 150_000), (3, 40_000), (2, 90_000), (5, 60_000)]
    gs = [Forest(d) for d, _ in specs]
    os_ = [OracleForest(d) for d, _ in specs]
    pts = [inputs.uniform_points(n, d, seed=730 + j) for j, (d, n) in enumerate(specs)]
    insert_batch(gs, [dev(p) for p in pts])
    for o, p in zip(os_, pts):
        o.insert(p)
    for j, (g, o) in enumerate(zip(gs, os_)):
        same_forest(g, o, "forest %d" % j)
    for g in gs:
        g.close()


def test_small_subtree_instance(monkeypatch):
    """Subtrees of fewer than 2,048 records go to the kernel's 256-thread
    instance when they are at least as many as the schedule's slots (two
    here): many small forests, of four dimensions, built in batched calls and
    rebuilt by an erase, tree by tree against the oracle; then k-NN rows
    (whose buffer trees are built the same way)."""
    from paper_2112_06188_gb300.forest import Forest, erase_batch, insert_batch, knn_batch
    from oracle.threads import oracle_knn
    monkeypatch.setenv("BDL_BUILD_SLOTS", "2")
    specs = [(d, n) for d in (2, 3, 5, 7) for n in (1_100, 2_500, 5_900)]
    gs = [Forest(d) for d, _ in specs]
    os_ = [OracleForest(d) for d, _ in specs]
    pts = [inputs.uniform_points(n, d, seed=740 + j) for j, (d, n) in enumerate(specs)]
    insert_batch(gs, [dev(p) for p in pts])
    for o, p in zip(os_, pts):
        o.insert(p)
    for j, (g, o) in enumerate(zip(gs, os_)):
        same_forest(g, o, "forest %d after the build" % j)
    eras = [inputs.sample_ids(np.arange(n), int(0.6 * n), seed=760 + j) for j, (_, n) in enumerate(specs)]
    erase_batch(gs, [dev(e) for e in eras])
    for o, e in zip(os_, eras):
        o.erase(e)
    for j, (g, o) in enumerate(zip(gs, os_)):
        same_forest(g, o, "forest %d after the erase" % j)
    qs = [inputs.uniform_points(600, d, seed=780 + j) for j, (d, _) in enumerate(specs)]
    out = knn_batch(gs, [dev(q) for q in qs], 6)
    torch.cuda.synchronize()
    for j, ((gi, gd), o, q) in enumerate(zip(out, os_, qs)):
        oi, od = oracle_knn(o, q, 6)
        assert np.array_equal(gi.cpu().numpy(), oi) and np.array_equal(gd.cpu().numpy(), od), "k-NN of forest %d" % j
    for g in gs:
        g.close()
