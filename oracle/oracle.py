"""ctypes binding of the serial CPU BDL-tree oracle (bdl_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and the
CPU-baseline / reference legs of bench.py.  The CUDA library never imports it.
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bdl_oracle.c")
_LIB = os.path.join(_HERE, "lib", "libbdl_oracle.so")
_lib = None

D2_NONE = np.iinfo(np.int64).max


def build(force=False):
    """Compile bdl_oracle.c into oracle/lib/libbdl_oracle.so (gcc, -O2)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + ".%d.tmp" % os.getpid()
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC",
                           "-o", tmp, _SRC])
    os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        i64, i32, u64 = ctypes.c_int64, ctypes.c_int, ctypes.c_uint64
        L.orc_forest_new.restype = P
        L.orc_forest_new.argtypes = [i32, i32, i32, i32, u64]
        L.orc_forest_free.argtypes = [P]
        L.orc_forest_set_split.restype = i32
        L.orc_forest_set_split.argtypes = [P, i32]
        L.orc_insert.restype = i64
        L.orc_insert.argtypes = [P, P, i64]
        L.orc_erase.restype = i64
        L.orc_erase.argtypes = [P, P, i64]
        L.orc_knn.argtypes = [P, P, i64, i32, P, P, P]
        L.orc_live_count.restype = i64
        L.orc_live_count.argtypes = [P]
        L.orc_tree_mask.restype = u64
        L.orc_tree_mask.argtypes = [P]
        L.orc_buffer.restype = i64
        L.orc_buffer.argtypes = [P, P, i64]
        L.orc_tree_info.restype = i32
        L.orc_tree_info.argtypes = [P, i32, P]
        L.orc_tree_nodes.restype = i32
        L.orc_tree_nodes.argtypes = [P, i32, P, P, P, P, P, P]
        L.orc_tree_leaves.restype = i32
        L.orc_tree_leaves.argtypes = [P, i32, P, P, P]
        L.orc_tree_bloom.restype = i32
        L.orc_tree_bloom.argtypes = [P, i32, P]
        L.orc_bloom_maybe.restype = i32
        L.orc_bloom_maybe.argtypes = [P, i32, ctypes.c_int32]
        L.orc_splitmix64.restype = u64
        L.orc_splitmix64.argtypes = [u64]
        L.orc_bruteforce_knn.argtypes = [i32, P, P, i64, P, i64, i32, P, P]
        _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def splitmix64(x):
    return int(lib().orc_splitmix64(ctypes.c_uint64(x & 0xFFFFFFFFFFFFFFFF)))


def bruteforce_knn(pts, ids, queries, k):
    """Exact k nearest neighbours of each query among (pts, ids) by (d2, id)."""
    pts = np.ascontiguousarray(pts, dtype=np.int32)
    ids = np.ascontiguousarray(ids, dtype=np.int32)
    q = np.ascontiguousarray(queries, dtype=np.int32)
    dim = q.shape[1]
    m = q.shape[0]
    out_ids = np.empty((m, k), dtype=np.int32)
    out_d2 = np.empty((m, k), dtype=np.int64)
    if m:
        lib().orc_bruteforce_knn(dim, _p(pts), _p(ids), len(ids), _p(q), m, k,
                                 _p(out_ids), _p(out_d2))
    return out_ids, out_d2


class OracleForest:
    """Serial BDL-tree: Insert_L / Erase_L / kNN_L of the paper, on the CPU."""

    def __init__(self, dim, leaf_size=16, buffer_size=1024, bloom_bits_per_key=16,
                 hash_seed=0x5EED, split="object"):
        """split: "object" (median of the points, the default) or "spatial"
        (midpoint of their extent), the two rules of Sec. V-C."""
        self.dim = dim
        self.leaf_size = leaf_size
        self.buffer_size = buffer_size
        self.split = split
        self._h = lib().orc_forest_new(dim, leaf_size, buffer_size,
                                       bloom_bits_per_key, hash_seed)
        if not self._h:
            raise ValueError("invalid oracle forest parameters")
        if split not in ("object", "spatial"):
            raise ValueError("split must be 'object' or 'spatial'")
        lib().orc_forest_set_split(self._h, 1 if split == "spatial" else 0)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().orc_forest_free(h)
            self._h = None

    def insert(self, pts):
        pts = np.ascontiguousarray(pts, dtype=np.int32).reshape(-1, self.dim)
        first = lib().orc_insert(self._h, _p(pts), len(pts))
        if first < 0:
            raise ValueError("coordinate outside [0, 2^20) or id space exhausted")
        return np.arange(first, first + len(pts), dtype=np.int32)

    def erase(self, ids):
        ids = np.ascontiguousarray(ids, dtype=np.int32)
        return int(lib().orc_erase(self._h, _p(ids), len(ids)))

    def knn(self, queries, k, stats=None):
        q = np.ascontiguousarray(queries, dtype=np.int32).reshape(-1, self.dim)
        m = len(q)
        out_ids = np.empty((m, k), dtype=np.int32)
        out_d2 = np.empty((m, k), dtype=np.int64)
        st = np.zeros(2, dtype=np.int64)
        if m:
            lib().orc_knn(self._h, _p(q), m, k, _p(out_ids), _p(out_d2), _p(st))
        if stats is not None:
            stats["nodes"] = int(st[0])
            stats["points"] = int(st[1])
        return out_ids, out_d2

    def size(self):
        return int(lib().orc_live_count(self._h))

    def tree_mask(self):
        return int(lib().orc_tree_mask(self._h))

    def buffer_ids(self):
        out = np.empty(self.buffer_size, dtype=np.int32)
        n = lib().orc_buffer(self._h, _p(out), len(out))
        return out[:n].copy()

    def tree_levels(self):
        F = self.tree_mask()
        return [i for i in range(64) if (F >> i) & 1]

    def tree(self, level):
        """Everything about static tree `level` as numpy arrays (vEB order)."""
        info = np.zeros(6, dtype=np.int64)
        if lib().orc_tree_info(self._h, level, _p(info)) != 0:
            return None
        size, live, h, nn, blocks = (int(x) for x in info[:5])
        d = self.dim
        key = np.empty(nn, np.int64)
        child = np.empty(2 * nn, np.int32)
        box = np.empty(nn * 2 * d, np.int32)
        nlive = np.empty(nn, np.int64)
        depth = np.empty(nn, np.int32)
        bfs = np.empty(nn, np.int64)
        lib().orc_tree_nodes(self._h, level, _p(key), _p(child), _p(box), _p(nlive),
                             _p(depth), _p(bfs))
        leaf_off = np.empty((1 << h) + 1, np.int64)
        ids = np.empty(size, np.int32)
        dead = np.empty(size, np.uint8)
        lib().orc_tree_leaves(self._h, level, _p(leaf_off), _p(ids), _p(dead))
        bloom = None
        if blocks:
            bloom = np.empty(blocks * 8, np.uint32)
            lib().orc_tree_bloom(self._h, level, _p(bloom))
        return dict(size=size, live=live, h=h, nnodes=nn, key=key,
                    child=child.reshape(nn, 2), box=box.reshape(nn, 2 * d),
                    node_live=nlive, depth=depth, bfs=bfs, leaf_off=leaf_off,
                    ids=ids, dead=dead.astype(bool), bloom=bloom)

    def bloom_maybe(self, level, pid):
        return int(lib().orc_bloom_maybe(self._h, level, int(pid)))
