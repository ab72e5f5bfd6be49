"""bdl_knn_noalloc: k-NN for callers that cannot allocate device memory while
they query (their free memory is held by another allocator, or the request
path must not wait on a pool).  Its scratch is a fixed array inside the
library; its rows must equal bdl_knn's, bit for bit, call after call, and the
oracle's.  Dimensions 2 and 5 use the largest query-ordering histogram the
array is sized for (2^20 bins); 3 and 7 smaller ones."""
import ctypes

import numpy as np
import pytest
import torch

from oracle.oracle import OracleForest
from paper_2112_06188_gb300 import inputs
from oracle.threads import oracle_knn

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2112_06188_gb300 import build_lib
    build_lib.build()


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def _knn(fn, f, q, k):
    from paper_2112_06188_gb300 import capi
    m = q.shape[0]
    oi = torch.full((m, k), -7, dtype=torch.int32, device="cuda")
    od = torch.full((m, k), -7, dtype=torch.int64, device="cuda")
    st = fn(f._h, _ptr(q), m, k, _ptr(oi), _ptr(od), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    capi.check(st, fn.__name__)
    torch.cuda.synchronize()
    return oi.cpu().numpy(), od.cpu().numpy()


def _forest(dim, n, seed):
    from paper_2112_06188_gb300.forest import Forest
    pts = inputs.uniform_points(n, dim, seed=seed)
    f, o = Forest(dim), OracleForest(dim)
    f.insert(torch.from_numpy(pts).cuda())
    o.insert(pts)
    era = inputs.sample_ids(np.arange(n), n // 8, seed=seed + 1)
    assert f.erase(torch.from_numpy(era).cuda()) == o.erase(era)
    return f, o, pts


@pytest.mark.parametrize("dim", [2, 3, 5])
def test_knn_noalloc_matches_knn(dim):
    from paper_2112_06188_gb300 import capi
    k = 10
    f, _, pts = _forest(dim, 300_000, seed=31 + dim)
    big = torch.from_numpy(inputs.queries_from(pts, 60_000, seed=33)).cuda()     # spatial order
    small = torch.from_numpy(inputs.uniform_points(2_000, dim, seed=34)).cuda()   # input order
    for q in (big, small):
        # the buffer tree is stale after the erase: the allocation-free call scans the buffer
        a1 = _knn(capi.bdl_knn_noalloc, f, q, k)
        ref = _knn(capi.bdl_knn, f, q, k)         # rebuilds the buffer tree
        a2 = _knn(capi.bdl_knn_noalloc, f, q, k)  # uses it
        for got in (a1, a2):
            assert np.array_equal(got[0], ref[0])
            assert np.array_equal(got[1], ref[1])
    f.close()


@pytest.mark.parametrize("dim", [2, 7])
def test_knn_noalloc_matches_oracle(dim):
    """Every row of two calls in a row (spatial order, then input order)
    against the oracle's kNN_L."""
    from paper_2112_06188_gb300 import capi
    k = 8
    f, o, pts = _forest(dim, 120_000, seed=41 + dim)
    for m, seed in ((40_000, 43), (3_000, 44)):
        qn = np.concatenate([inputs.queries_from(pts, m // 2, seed=seed),
                             inputs.uniform_points(m - m // 2, dim, seed=seed + 1)])
        q = torch.from_numpy(np.ascontiguousarray(qn)).cuda()
        gi, gd = _knn(capi.bdl_knn_noalloc, f, q, k)
        oi, od = oracle_knn(o, qn, k)
        assert np.array_equal(gi, oi)
        assert np.array_equal(gd, od)
    f.close()


def test_knn_noalloc_rejects_over_limit():
    """Over the stated maximum: rejected on the host before any device work
    (NULL buffers, so that a regression of the check would still stop at the
    pointer check instead of writing anywhere)."""
    from paper_2112_06188_gb300 import capi
    f, _, _ = _forest(3, 5_000, seed=51)
    m = (1 << 20) + 1
    st = capi.load().bdl_knn_noalloc(f._h, None, m, 10, None, None, None)
    assert st == capi.BDL_EINVAL
    assert "1,048,576" in capi.last_error()
    f.close()
