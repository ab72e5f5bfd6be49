"""Batched forests through bdl_insert_batch / bdl_erase_batch / bdl_knn_batch.

One call on many independent forests must give every forest exactly what the
single-forest calls give (same trees, node for node, same buffers, same bloom
words, same k-NN rows), and what the oracle gives.  The workload is many small
forests of log-uniform sizes in 2-D and 3-D with insert batches of 5-20%,
delete batches of 2-10% (some far larger, so that trees fall below half and
are rebuilt) and k = 8 queries per forest.
"""
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


def log_uniform(n, lo, hi, seed):
    r = np.random.default_rng(seed)
    return np.exp(r.uniform(np.log(lo), np.log(hi), size=n)).astype(np.int64)


def same_state(a, b, what):
    """Two forests (GPU/GPU or GPU/oracle) hold the same structure."""
    assert a.tree_mask() == b.tree_mask(), what
    assert np.array_equal(np.sort(a.buffer_ids()), np.sort(b.buffer_ids())), what
    assert a.size() == b.size(), what
    for lvl in b.tree_levels():
        ta, tb = a.tree(lvl), b.tree(lvl)
        assert_same_tree(ta, tb, "%s tree %d" % (what, lvl))
        assert (ta["bloom"] is None) == (tb["bloom"] is None), what
        if ta["bloom"] is not None:
            assert np.array_equal(ta["bloom"], tb["bloom"]), "%s bloom %d" % (what, lvl)


class Workload:
    """nf forests, a live set per forest, seeded batches."""

    def __init__(self, nf, lo, hi, dims, seed, configs=None):
        from paper_2112_06188_gb300.forest import Forest
        self.rng = np.random.default_rng(seed)
        self.sizes = log_uniform(nf, lo, hi, seed)
        self.dims = [dims[i % len(dims)] for i in range(nf)]
        self.configs = configs or [dict(leaf_size=16, buffer_size=1024)] * nf
        self.A = [Forest(d, **c) for d, c in zip(self.dims, self.configs)]   # batched calls
        self.B = [Forest(d, **c) for d, c in zip(self.dims, self.configs)]   # single calls
        self.live = [inputs.LiveSet(d) for d in self.dims]

    def points(self, i, n):
        return self.rng.integers(0, 1 << 20, size=(n, self.dims[i]), dtype=np.int32)

    def close(self):
        for f in self.A + self.B:
            f.close()


def run_insert(w, pts):
    from paper_2112_06188_gb300.forest import insert_batch
    ids_a = insert_batch(w.A, [dev(p) for p in pts])
    for i, p in enumerate(pts):
        ids_b = w.B[i].insert(dev(p))
        want = w.live[i].insert(p)
        assert np.array_equal(ids_a[i].cpu().numpy(), want)
        assert np.array_equal(ids_b.cpu().numpy(), want)


def run_erase(w, ids):
    from paper_2112_06188_gb300.forest import erase_batch
    na = erase_batch(w.A, [dev(e) for e in ids])
    for i, e in enumerate(ids):
        nb = w.B[i].erase(dev(e))
        assert na[i] == nb == w.live[i].erase(e)


def run_knn(w, k, m_lo, m_hi):
    from paper_2112_06188_gb300.forest import knn_batch
    qs = []
    for i in range(len(w.A)):
        m = int(w.rng.integers(m_lo, m_hi + 1))
        lp = w.live[i].coords[w.live[i].alive]
        q = inputs.queries_from(lp, m, seed=int(w.rng.integers(1 << 30))) if len(lp) else w.points(i, m)
        qs.append(q)
    out = knn_batch(w.A, [dev(q) for q in qs], k)
    rows = []
    for i, q in enumerate(qs):
        bi, bd = w.B[i].knn(dev(q), k)
        ai, ad = out[i]
        assert torch.equal(ai, bi) and torch.equal(ad, bd), "forest %d" % i
        rows.append((q, ai.cpu().numpy(), ad.cpu().numpy()))
    return rows


def test_batch_equals_single_calls_and_oracle():
    nf = 24
    w = Workload(nf, 500, 60000, dims=(2, 3), seed=11)
    ora = {i: OracleForest(w.dims[i], leaf_size=16, buffer_size=1024) for i in range(0, nf, 6)}

    def check(tag):
        for i in range(nf):
            same_state(w.A[i], w.B[i], "%s forest %d" % (tag, i))
        for i, o in ora.items():
            same_state(w.A[i], o, "%s forest %d vs oracle" % (tag, i))

    pts = [w.points(i, int(w.sizes[i])) for i in range(nf)]
    run_insert(w, pts)
    for i, o in ora.items():
        o.insert(pts[i])
    check("build")
    for step in range(3):
        frac = w.rng.uniform(0.05, 0.20, size=nf)
        pts = [w.points(i, max(1, int(frac[i] * w.sizes[i]))) for i in range(nf)]
        run_insert(w, pts)
        for i, o in ora.items():
            o.insert(pts[i])
        dfrac = w.rng.uniform(0.02, 0.10, size=nf)
        if step == 1:
            dfrac[::4] = 0.6          # these fall below half: rebuilds in several forests at once
        ids = []
        for i in range(nf):
            lid = w.live[i].live_ids()
            ids.append(inputs.sample_ids(lid, max(1, int(dfrac[i] * len(lid))), seed=100 * step + i))
        for i, o in ora.items():
            assert o.erase(ids[i]) == int(np.isin(ids[i], w.live[i].live_ids()).sum())
        run_erase(w, ids)
        check("step %d" % step)
        rows = run_knn(w, 8, 1000, 5000)
        for i, o in ora.items():
            q, gi, gd = rows[i]
            oi, od = o.knn(q, 8)
            assert np.array_equal(gi, oi) and np.array_equal(gd, od), "forest %d vs oracle" % i
    w.close()


def test_batch_mixed_dims_and_configs():
    """Forests of dimensions 2, 3, 5 and 7, different leaf sizes, buffer sizes and
    bloom seeds in the same calls."""
    configs = [dict(leaf_size=16, buffer_size=1024), dict(leaf_size=8, buffer_size=512, hash_seed=7),
               dict(leaf_size=32, buffer_size=2048, bloom_bits_per_key=8),
               dict(leaf_size=4, buffer_size=256, hash_seed=123456789)]
    nf = 12
    w = Workload(nf, 300, 30000, dims=(2, 3, 5, 7), seed=5,
                 configs=[configs[i % 4] for i in range(nf)])
    run_insert(w, [w.points(i, int(w.sizes[i])) for i in range(nf)])
    for step in range(2):
        ids = [inputs.sample_ids(w.live[i].live_ids(), max(1, len(w.live[i].live_ids()) // 3),
                                 seed=step * 50 + i) for i in range(nf)]
        run_erase(w, ids)
        run_insert(w, [w.points(i, int(w.sizes[i]) // 7 + 1) for i in range(nf)])
        for i in range(nf):
            same_state(w.A[i], w.B[i], "forest %d" % i)
        run_knn(w, 5, 1, 700)
    w.close()


def test_batch_erase_where_some_forests_erase_nothing():
    """In one erase batch, the forests whose ids are all dead or absent are left
    exactly as their single calls leave them (lazy blooms still unbuilt), while
    the others erase, including some already erased ids again."""
    nf = 8
    w = Workload(nf, 2000, 20000, dims=(2, 3), seed=17)
    run_insert(w, [w.points(i, int(w.sizes[i])) for i in range(nf)])
    for step in range(2):
        ids = []
        for i in range(nf):
            lid = w.live[i].live_ids()
            n_ids = len(w.live[i].alive)
            if (i + step) % 2:
                ids.append(np.array([n_ids + 10, -5, n_ids + 10, n_ids], np.int32))
            else:
                ids.append(inputs.sample_ids(lid, len(lid) // 5, seed=10 * step + i))
        run_erase(w, ids)
        for i in range(nf):
            same_state(w.A[i], w.B[i], "step %d forest %d" % (step, i))
        run_erase(w, ids)             # the same batches again: nothing left to erase
        for i in range(nf):
            same_state(w.A[i], w.B[i], "step %d again, forest %d" % (step, i))
        run_knn(w, 6, 100, 2000)
    w.close()


def test_batch_large_queries_sorted_path():
    """Query batches above the spatial-sort threshold in some forests, below it in others."""
    w = Workload(4, 40000, 120000, dims=(3,), seed=9)
    run_insert(w, [w.points(i, int(w.sizes[i])) for i in range(4)])
    run_knn(w, 10, 20000, 50000)
    w.close()


def test_batch_all_or_nothing_on_bad_coordinate():
    from paper_2112_06188_gb300 import capi
    from paper_2112_06188_gb300.forest import insert_batch
    w = Workload(3, 2000, 5000, dims=(2,), seed=3)
    run_insert(w, [w.points(i, int(w.sizes[i])) for i in range(3)])
    before = [(f.tree_mask(), f.size(), list(f.buffer_ids())) for f in w.A]
    pts = [w.points(i, 3000) for i in range(3)]
    pts[2][1234, 1] = 1 << 20
    with pytest.raises(capi.BdlError) as e:
        insert_batch(w.A, [dev(p) for p in pts])
    assert e.value.status == capi.BDL_EINVAL
    assert [(f.tree_mask(), f.size(), list(f.buffer_ids())) for f in w.A] == before
    pts[2][1234, 1] = 5
    run_insert(w, pts)                 # ids continue where they were
    for i in range(3):
        same_state(w.A[i], w.B[i], "forest %d" % i)
    w.close()


def test_batch_argument_rules():
    from paper_2112_06188_gb300 import capi
    from paper_2112_06188_gb300.forest import Forest, erase_batch, insert_batch, knn_batch
    f, g = Forest(2), Forest(2)
    p = dev(inputs.uniform_points(3000, 2, seed=1))
    with pytest.raises(capi.BdlError):
        insert_batch([f, f], [p, p])
    assert f.size() == 0
    insert_batch([f, g], [p, p[:100]])
    with pytest.raises(capi.BdlError):
        erase_batch([g, g], [dev(np.arange(5, dtype=np.int32))] * 2)
    assert g.size() == 100
    # the same forest twice in a k-NN batch is allowed
    q = dev(inputs.uniform_points(50, 2, seed=2))
    (a_i, a_d), (b_i, b_d) = knn_batch([f, f], [q, q[:7]], 4)
    s_i, s_d = f.knn(q, 4)
    assert torch.equal(a_i, s_i) and torch.equal(b_i, s_i[:7]) and torch.equal(b_d, s_d[:7])
    # empty batches and empty entries
    assert insert_batch([], []) == []
    assert erase_batch([f, g], [dev(np.zeros(0, np.int32)), dev(np.array([3, 3, -1], np.int32))]) == [0, 1]
    out = knn_batch([f, g], [dev(np.zeros((0, 2), np.int32)), q], 3)
    assert out[0][0].shape == (0, 3)
    assert torch.equal(out[1][0], g.knn(q, 3)[0])
    f.close()
    g.close()


def test_knn_plan_launch_and_graph():
    """A prepared k-NN: equal to bdl_knn_batch, follows new query contents,
    replays from a CUDA graph, refuses to run after an update."""
    from paper_2112_06188_gb300 import capi
    from paper_2112_06188_gb300.forest import Forest, KnnPlan, knn_batch
    dims = [2, 3, 3, 5, 2]
    F = [Forest(d) for d in dims]
    for i, (f, d) in enumerate(zip(F, dims)):
        f.insert(dev(inputs.uniform_points(4000 + 9000 * i, d, seed=i)))
    ms = [100, 1, 40000, 2500, 0]            # one batch above the spatial-sort threshold
    qs = [dev(inputs.uniform_points(m, d, seed=10 + i)) for i, (m, d) in enumerate(zip(ms, dims))]
    plan = KnnPlan(F, qs, 6)
    got = plan.launch()
    want = knn_batch(F, qs, 6)
    for (a, b), (c, d) in zip(got, want):
        assert torch.equal(a, c) and torch.equal(b, d)
    # new contents, same tensors
    for i, (q, d) in enumerate(zip(qs, dims)):
        q.copy_(dev(inputs.uniform_points(q.shape[0], d, seed=50 + i)))
    got = [(a.clone(), b.clone()) for a, b in plan.launch()]
    want = knn_batch(F, qs, 6)
    for (a, b), (c, d) in zip(got, want):
        assert torch.equal(a, c) and torch.equal(b, d)
    # captured once, replayed with fresh queries
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        plan.launch(stream=s)
    for i, (q, d) in enumerate(zip(qs, dims)):
        q.copy_(dev(inputs.uniform_points(q.shape[0], d, seed=90 + i)))
    for o in plan.out:
        o[0].fill_(-7)
    g.replay()
    torch.cuda.synchronize()
    want = knn_batch(F, qs, 6)
    for (a, b), (c, d) in zip(plan.out, want):
        assert torch.equal(a, c) and torch.equal(b, d)
    # an update invalidates the plan
    F[1].insert(dev(inputs.uniform_points(10, 3, seed=1)))
    with pytest.raises(capi.BdlError):
        plan.launch()
    plan.close()
    for f in F:
        f.close()
