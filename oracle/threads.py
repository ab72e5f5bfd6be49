"""The oracle's k-NN calls over chunks of queries in host threads.

TEST INFRASTRUCTURE ONLY, like the rest of oracle/: used by tests/ and by the
CPU legs of bench.py.

OracleForest.knn and bruteforce_knn only read the forest or the point set,
allocate their scratch per call, and release the GIL while they run (ctypes
foreign calls), so disjoint chunks of a query batch can go to separate
threads.  This changes nothing in what the oracle computes -- every row is
the same serial computation -- only how many rows run at once, so that
row-by-row parity on batches of tens of thousands of queries (the sizes at
which the CUDA path puts queries in spatial order) fits in a test.
"""
import concurrent.futures as cf
import os

import numpy as np

from .oracle import bruteforce_knn


def _threads():
    return max(1, min(32, os.cpu_count() or 1))


def _chunked(fn, q, k, threads):
    q = np.ascontiguousarray(q)
    m = len(q)
    threads = threads or _threads()
    step = max(1, -(-m // (4 * threads)))
    bounds = [(a, min(m, a + step)) for a in range(0, m, step)]
    out_i = np.empty((m, k), dtype=np.int32)
    out_d = np.empty((m, k), dtype=np.int64)

    def run(ab):
        a, b = ab
        out_i[a:b], out_d[a:b] = fn(q[a:b])

    with cf.ThreadPoolExecutor(max_workers=threads) as ex:
        list(ex.map(run, bounds))
    return out_i, out_d


def oracle_knn(o, q, k, threads=None):
    """OracleForest o's kNN_L rows for queries q, computed in `threads` threads."""
    return _chunked(lambda qq: o.knn(qq, k), q, k, threads)


def bruteforce_knn_threads(pts, ids, q, k, threads=None):
    """bruteforce_knn(pts, ids, q, k), with the queries split over threads."""
    pts = np.ascontiguousarray(pts, dtype=np.int32)
    ids = np.ascontiguousarray(ids, dtype=np.int32)
    return _chunked(lambda qq: bruteforce_knn(pts, ids, qq, k), q, k, threads)
