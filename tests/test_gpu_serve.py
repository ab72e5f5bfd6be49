"""The request server (bdl_server_*): every request's result in the mix --
requests arriving while others run, batched as they come -- equals its result
alone, i.e. the plain calls issued one by one in submission order; and those
are the oracle's (the plain path is pinned in test_gpu_parity.py; here a
sample of rows is also checked against brute force)."""
import threading
import time

import numpy as np
import pytest
import torch

from oracle.oracle import bruteforce_knn
from paper_2112_06188_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2112_06188_gb300 import build_lib
    build_lib.build()


def stream_of(n_req, seed, dim=5, n0=100_000):
    w = inputs.ServeWorkload(dim=dim, n0=n0, n_final=10 ** 9, rate=2000.0, seed=seed,
                             ins=(500, 60_000), dele=(500, 20_000), knn=(1, 6_000),
                             max_requests=n_req)
    return w.initial, list(w.requests())


def alone(dim, initial, reqs):
    """The plain path: each request by itself, in order."""
    from paper_2112_06188_gb300.forest import Forest
    f = Forest(dim)
    f.insert(torch.from_numpy(initial).cuda())
    out = []
    for _, kind, payload, k in reqs:
        x = torch.from_numpy(payload).cuda()
        if kind == "insert":
            try:
                out.append(("insert", f.insert(x).cpu().numpy()))
            except Exception as e:
                out.append(("insert", getattr(e, "status", -1)))
        elif kind == "erase":
            out.append(("erase", f.erase(x)))
        else:
            gi, gd = f.knn(x, k)
            out.append(("knn", (gi.cpu().numpy(), gd.cpu().numpy())))
    f.close()
    return out


def in_mix(dim, initial, reqs, paced=True, **server_kw):
    """The same requests through the server, submitted at their arrival times
    (paced) or all at once, from a thread of their own."""
    from paper_2112_06188_gb300.forest import Forest
    from paper_2112_06188_gb300.serve import Server
    f = Forest(dim)
    f.insert(torch.from_numpy(initial).cuda())
    torch.cuda.synchronize()
    s = Server(f, **server_kw)
    tickets = [None] * len(reqs)
    payloads = [torch.from_numpy(np.ascontiguousarray(p)).pin_memory() for _, _, p, _ in reqs]

    def submitter():
        t0 = time.perf_counter()
        for i, ((t, kind, _, k), payload) in enumerate(zip(reqs, payloads)):
            if paced:
                dt = t - (time.perf_counter() - t0)
                if dt > 0:
                    time.sleep(dt)
            if kind == "insert":
                tickets[i] = s.insert(payload)
            elif kind == "erase":
                tickets[i] = s.erase(payload)
            else:
                tickets[i] = s.knn(payload, k)

    th = threading.Thread(target=submitter)
    th.start()
    th.join()
    res = [s.wait(t) for t in tickets]
    groups = s.groups()
    s.close()
    size = f.size()
    f.close()
    return res, groups, size


def compare(reqs, ref, res):
    from paper_2112_06188_gb300 import capi
    for i, ((_, kind, payload, k), r, got) in enumerate(zip(reqs, ref, res)):
        assert r[0] == kind
        if kind == "insert":
            if isinstance(r[1], int):
                assert got["status"] == r[1] == capi.BDL_EINVAL, i
            else:
                assert got["status"] == 0, i
                assert np.array_equal(got["ids"].numpy(), r[1]), i
        elif kind == "erase":
            assert got["status"] == 0 and got["n_done"] == r[1], i
        else:
            assert got["status"] == 0, i
            assert np.array_equal(got["ids"].numpy(), r[1][0]), "k-NN ids of request %d" % i
            assert np.array_equal(got["d2"].numpy(), r[1][1]), "k-NN d2 of request %d" % i


def test_mix_equals_alone():
    dim = 5
    initial, reqs = stream_of(120, seed=1, dim=dim)
    ref = alone(dim, initial, reqs)
    res, groups, _ = in_mix(dim, initial, reqs, paced=True)
    compare(reqs, ref, res)
    assert groups <= len(reqs)
    # every request's timestamps are ordered
    for r in res:
        assert r["t_submit_ms"] <= r["t_start_ms"] <= r["t_done_ms"]


def test_burst_is_batched_and_equal():
    """All requests at once: consecutive k-NN runs and insert runs share launches."""
    dim = 3
    initial, reqs = stream_of(150, seed=2, dim=dim, n0=50_000)
    ref = alone(dim, initial, reqs)
    res, groups, _ = in_mix(dim, initial, reqs, paced=False)
    compare(reqs, ref, res)
    # at least one device group per run of same-kind requests, and fewer groups
    # than requests once runs merge
    kinds = [k for _, k, _, _ in reqs]
    runs = 1 + sum(1 for a, b in zip(kinds, kinds[1:]) if a != b)
    assert runs <= groups < len(reqs)


def test_erase_runs_merge_with_exact_counts():
    """A burst of erases that overlap (the same id in several requests,
    repeated inside one request, dead, negative and never-inserted ids) runs
    as merged Erase_L calls; every request's count is the one it gets when
    the erases run one after another, and the forest ends the same."""
    dim = 3
    n0 = 40_000
    initial = inputs.uniform_points(n0, dim, seed=11)
    rng = np.random.default_rng(12)
    reqs = []
    for j in range(12):
        ids = rng.integers(0, n0, size=int(rng.integers(100, 3_000))).astype(np.int32)
        if j % 3 == 0 and reqs:
            ids = np.concatenate([ids, reqs[-1][2][:50]])          # overlaps the previous request
        ids = np.concatenate([ids, ids[:10], np.array([-1, n0 + 5, 2**31 - 1], np.int32)])
        reqs.append((0.0, "erase", ids.astype(np.int32), 0))
    q = inputs.uniform_points(2_000, dim, seed=13)
    reqs.append((0.0, "knn", q, 9))
    ref = alone(dim, initial, reqs)
    res, groups, _ = in_mix(dim, initial, reqs, paced=False)
    compare(reqs, ref, res)
    assert groups < len(reqs)
    counts = [r["n_done"] for r in res[:-1]]
    live = inputs.LiveSet(dim)
    live.insert(initial)
    assert counts == [live.erase(p) for _, _, p, _ in reqs[:-1]]


def test_knn_runs_mix_k():
    """Small k-NN requests with k in {1, 5, 10, 32} submitted together share
    launches; each request's rows are its own k's rows."""
    dim = 2
    initial = inputs.uniform_points(30_000, dim, seed=21)
    rng = np.random.default_rng(22)
    reqs = [(0.0, "knn", inputs.uniform_points(int(rng.integers(1, 2_000)), dim, seed=30 + j),
             int(rng.choice([1, 5, 10, 32]))) for j in range(40)]
    ref = alone(dim, initial, reqs)
    res, groups, _ = in_mix(dim, initial, reqs, paced=False)
    compare(reqs, ref, res)
    assert groups < len(reqs) // 2


def test_serial_mode_and_small_budget():
    dim = 2
    initial, reqs = stream_of(60, seed=3, dim=dim, n0=30_000)
    ref = alone(dim, initial, reqs)
    res, groups, _ = in_mix(dim, initial, reqs, paced=False, serial=True)
    compare(reqs, ref, res)
    assert groups == len(reqs)
    # a staging budget far below one request: each still runs (alone when too big)
    res, groups, _ = in_mix(dim, initial, reqs, paced=False, staging_budget_bytes=4096, max_inflight=3)
    compare(reqs, ref, res)


def test_bad_insert_in_a_merged_run():
    dim = 3
    initial, reqs = stream_of(40, seed=4, dim=dim, n0=20_000)
    reqs = [r for r in reqs if r[1] != "knn"][:10]
    bad = [i for i, r in enumerate(reqs) if r[1] == "insert"][1]
    p = reqs[bad][2].copy()
    p[len(p) // 2, 0] = -5
    reqs[bad] = (reqs[bad][0], "insert", p, 0)
    # queries after the run see the same state
    q = inputs.uniform_points(300, dim, seed=9)
    reqs.append((reqs[-1][0], "knn", q, 7))
    ref = alone(dim, initial, reqs)
    res, _, _ = in_mix(dim, initial, reqs, paced=False)
    compare(reqs, ref, res)
    # and the final k-NN rows are the exact answer on the live set
    live = inputs.LiveSet(dim)
    live.insert(initial)
    for (_, kind, payload, _), r in zip(reqs, res):
        if kind == "insert" and r["status"] == 0:
            live.insert(payload)
        elif kind == "erase":
            live.erase(payload)
    lp, lid = live.live_points()
    bi, bd = bruteforce_knn(lp, lid, q[:40], 7)
    assert np.array_equal(res[-1]["ids"].numpy()[:40], bi)
    assert np.array_equal(res[-1]["d2"].numpy()[:40], bd)
