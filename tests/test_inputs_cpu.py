"""The seeded synthetic workloads (CPU): reproducible, on the grid, and shaped
as stated -- batched forests of log-uniform sizes with 5-20% inserts and
2-10% deletes of live ids, and a Poisson request stream whose erases only
name live ids."""
import numpy as np

from paper_2112_06188_gb300 import inputs


def test_forests_workload_shape_and_reproducibility():
    a = inputs.ForestsWorkload(nf=64, lo=1000, hi=200000, seed=4)
    b = inputs.ForestsWorkload(nf=64, lo=1000, hi=200000, seed=4)
    assert np.array_equal(a.sizes, b.sizes) and a.dims == b.dims
    assert a.sizes.min() >= 1000 and a.sizes.max() <= 200000
    assert set(a.dims) <= {2, 3}
    for p, n, d in zip(a.initial, a.sizes, a.dims):
        assert p.shape == (n, d) and p.min() >= 0 and p.max() < inputs.GRID
    live_before = [int(x.sum()) for x in a.alive]
    sa, sb = a.step(), b.step()
    for i, ((ins, era, q), (ins2, era2, q2)) in enumerate(zip(sa, sb)):
        assert np.array_equal(ins, ins2) and np.array_equal(era, era2) and np.array_equal(q, q2)
        assert 0.05 * a.sizes[i] - 1 <= len(ins) <= 0.20 * a.sizes[i] + 1
        live = live_before[i] + len(ins)
        assert 0.02 * live - 1 <= len(era) <= 0.10 * live + 1
        assert len(np.unique(era)) == len(era)
        assert not a.alive[i][era].any()            # erased after the step
        assert 1000 <= len(q) <= 5000 and q.shape[1] == a.dims[i]


def test_serve_workload_stream():
    w = inputs.ServeWorkload(dim=5, n0=20000, n_final=10 ** 9, rate=500.0, seed=5,
                             ins=(100, 5000), dele=(100, 3000), knn=(1, 2000), max_requests=400)
    alive = np.ones(20000, dtype=bool)
    t_prev, kinds = 0.0, []
    for t, kind, payload, k in w.requests():
        assert t > t_prev
        t_prev = t
        kinds.append(kind)
        if kind == "insert":
            assert payload.shape[1] == 5 and 100 <= len(payload) <= 5000
            alive = np.concatenate([alive, np.ones(len(payload), dtype=bool)])
        elif kind == "erase":
            assert alive[payload].all() and len(np.unique(payload)) == len(payload)
            alive[payload] = False
        else:
            assert k in (1, 5, 10) and 1 <= len(payload) <= 2000
    assert len(kinds) == 400
    frac = np.array([kinds.count(x) for x in ("insert", "erase", "knn")]) / len(kinds)
    assert np.all(np.abs(frac - np.array([0.4, 0.1, 0.5])) < 0.08)
    assert 0.4 < t_prev < 1.4        # ~400 arrivals at 500 per second
