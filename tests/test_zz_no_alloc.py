"""bdl_knn_noalloc: k-NN for callers that cannot allocate device memory while
they query (their free memory is held by another allocator, or the request
path must not wait on a pool).  Its scratch is a fixed array inside the
library; its rows must equal bdl_knn's, bit for bit, call after call."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2112_06188_gb300 import inputs

pytestmark = pytest.mark.gpu


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


def test_knn_noalloc_matches_knn():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2112_06188_gb300 import build_lib, capi
    build_lib.build()
    from paper_2112_06188_gb300.forest import Forest

    dim, k = 3, 10
    pts = inputs.uniform_points(300_000, dim, seed=31)
    f = Forest(dim)
    f.insert(torch.from_numpy(pts).cuda())
    f.erase(torch.from_numpy(inputs.sample_ids(np.arange(300_000), 40_000, seed=32)).cuda())
    big = torch.from_numpy(inputs.queries_from(pts, 60_000, seed=33)).cuda()     # ordered path
    small = torch.from_numpy(inputs.uniform_points(2_000, dim, seed=34)).cuda()   # input order

    for q in (big, small):
        # the buffer tree is stale after the erase: the allocation-free call scans the buffer
        a1 = _knn(capi.bdl_knn_noalloc, f, q, k)
        ref = _knn(capi.bdl_knn, f, q, k)         # rebuilds the buffer tree
        a2 = _knn(capi.bdl_knn_noalloc, f, q, k)  # uses it
        for got in (a1, a2):
            assert np.array_equal(got[0], ref[0])
            assert np.array_equal(got[1], ref[1])

    # over the stated maximum: rejected before any device work
    m = (1 << 20) + 1
    st = capi.load().bdl_knn_noalloc(f._h, _ptr(small), m, k, _ptr(small), _ptr(small), None)
    assert st == capi.BDL_EINVAL
    assert "1,048,576" in capi.last_error()
    f.close()
