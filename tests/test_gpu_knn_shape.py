"""The k-NN kernel's launch shape (threads per block, queries per warp) is a
speed knob only: every shape must give the rows of kNN_L (Alg. 5) bit for
bit.  Each shape is compared row by row with the oracle on the sorted path
(>= 2^15 queries, spatial order) and the input-order path, at k = 10 and at
k = 32 (where a 256-thread block is halved to fit its top-k slots), through
the single-forest call, the batched call (which launches with the first
forest's shape) and a prepared plan (which keeps the shape it was made
with)."""
import numpy as np
import pytest
import torch

from oracle.oracle import OracleForest
from oracle.threads import oracle_knn
from paper_2112_06188_gb300 import inputs

pytestmark = pytest.mark.gpu

SHAPES = [(b, q) for b in (64, 128, 256) for q in (32, 64, 128)]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2112_06188_gb300 import build_lib
    build_lib.build()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def assert_rows(got, want, what):
    gi, gd = (x.cpu().numpy() for x in got)
    oi, od = want
    bad = (gi != oi).any(1) | (gd != od).any(1)
    assert not bad.any(), "%s: %d of %d rows differ" % (what, int(bad.sum()), len(bad))


def forest_pair(dim, n0, seed):
    """GPU forest and oracle after a build, an insert and an erase that
    rebuilds trees."""
    from paper_2112_06188_gb300.forest import Forest
    pts = inputs.uniform_points(n0, dim, seed=seed)
    g, o = Forest(dim), OracleForest(dim)
    live = inputs.LiveSet(dim)
    for x in (g, o, live):
        x.insert(pts if x is not g else dev(pts))
    more = inputs.uniform_points(n0 // 5 + 77, dim, seed=seed + 1)
    for x in (g, o, live):
        x.insert(more if x is not g else dev(more))
    era = inputs.sample_ids(live.live_ids(), int(0.55 * live.alive.sum()), seed=seed + 2)
    assert g.erase(dev(era)) == o.erase(era) == live.erase(era)
    lp, _ = live.live_points()
    return g, o, lp


@pytest.mark.parametrize("k", [10, 32])
def test_every_shape_matches_oracle(k):
    g, o, lp = forest_pair(3, 200_000, seed=500 + k)
    big = np.concatenate([inputs.queries_from(lp, 20_000, seed=510),
                          inputs.uniform_points(20_000, 3, seed=511)])       # sorted path
    small = inputs.uniform_points(2_500, 3, seed=512)                        # input order
    for q in (big, small):
        want = oracle_knn(o, q, k)
        qd = dev(q)
        for sh in SHAPES:
            g.set_knn_shape(*sh)
            assert_rows(g.knn(qd, k), want, "shape %s, m=%d, k=%d" % (sh, len(q), k))
    g.close()


def test_batched_and_plan_use_first_forest_shape():
    from paper_2112_06188_gb300.forest import KnnPlan, knn_batch
    pairs = [forest_pair(2, 60_000, seed=520), forest_pair(2, 30_000, seed=530), forest_pair(5, 40_000, seed=540)]
    k = 8
    qs = [np.concatenate([inputs.queries_from(lp, 20_000, seed=550 + j), inputs.uniform_points(15_000, g.dim, seed=560 + j)])
          if j == 0 else inputs.uniform_points(3_000 + 500 * j, g.dim, seed=560 + j)
          for j, (g, _, lp) in enumerate(pairs)]
    wants = [oracle_knn(o, q, k) for (_, o, _), q in zip(pairs, qs)]
    gs = [g for g, _, _ in pairs]
    qd = [dev(q) for q in qs]
    for sh in ((64, 128), (256, 64), (128, 32)):
        gs[0].set_knn_shape(*sh)
        out = knn_batch(gs, qd, k)
        torch.cuda.synchronize()
        for j, (got, want) in enumerate(zip(out, wants)):
            assert_rows(got, want, "batched, shape %s, forest %d" % (sh, j))
    # a plan made under one shape keeps it after the forest's shape changes
    gs[0].set_knn_shape(256, 128)
    plan = KnnPlan(gs, qd, k)
    gs[0].set_knn_shape(64, 32)
    plan.launch()
    torch.cuda.synchronize()
    for j, want in enumerate(wants):
        assert_rows(plan.out[j], want, "plan, forest %d" % j)
    plan.close()
    for g in gs:
        g.close()


def test_shape_values_checked():
    from paper_2112_06188_gb300 import capi
    g, _, _ = forest_pair(3, 5_000, seed=570)
    L = capi.load()
    for b, q in ((96, 32), (512, 32), (128, 16), (128, 256), (-1, 32)):
        assert L.bdl_set_knn_shape(g._h, b, q) == capi.BDL_EINVAL
    assert L.bdl_set_knn_shape(g._h, 0, 0) == capi.BDL_OK          # the defaults
    g.close()


def test_default_device_accepts_current_device_outputs():
    """A forest made without a device index lives on the current device, and
    output buffers there (cuda:N) are accepted."""
    from paper_2112_06188_gb300.forest import Forest
    g, o, lp = forest_pair(2, 5_000, seed=580)
    h = Forest(2)
    assert h.device == torch.device("cuda", torch.cuda.current_device())
    h.insert(dev(lp))
    q = inputs.uniform_points(100, 2, seed=581)
    n = torch.cuda.current_device()
    out = (torch.empty((100, 4), dtype=torch.int32, device="cuda:%d" % n),
           torch.empty((100, 4), dtype=torch.int64, device="cuda:%d" % n))
    h.knn(dev(q), 4, out=out)
    g.close()
    h.close()


def test_batched_call_at_k32():
    """The table-driven kernel at the largest k: its top-k slots fill 48 KB
    of shared memory at 128 threads, with the warps' job and tree slots on
    top (the launch opts in to the larger size)."""
    from paper_2112_06188_gb300.forest import knn_batch
    pairs = [forest_pair(3, 40_000, seed=590), forest_pair(3, 20_000, seed=591)]
    qs = [inputs.uniform_points(2_000 + 700 * j, 3, seed=592 + j) for j in range(2)]
    out = knn_batch([g for g, _, _ in pairs], [dev(q) for q in qs], 32)
    torch.cuda.synchronize()
    for j, ((g, o, _), q) in enumerate(zip(pairs, qs)):
        assert_rows(out[j], oracle_knn(o, q, 32), "k=32 batched, forest %d" % j)
    for g, _, _ in pairs:
        g.close()
