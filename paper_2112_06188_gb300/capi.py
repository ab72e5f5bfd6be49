"""ctypes binding of the C ABI in include/bdl.h -- argument marshalling only.

Every function here has the name of the C entry point it calls and takes the
same arguments (device pointers as Python ints, the stream as an int handle);
all computation happens in the CUDA library.  Loading fails loudly if the
library has not been built: there is no fallback.
"""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "lib", "libbdl_gb300.so")

BDL_OK, BDL_EINVAL, BDL_ENOMEM, BDL_ECUDA, BDL_ETIMEOUT, BDL_EINTERNAL = range(6)

SYMBOLS = [
    "bdl_default_config", "bdl_create", "bdl_insert", "bdl_erase", "bdl_knn", "bdl_size",
    "bdl_destroy", "bdl_status_string", "bdl_last_error", "bdl_tree_mask", "bdl_buffer_ids",
    "bdl_tree_info", "bdl_tree_export", "bdl_bloom_export", "bdl_knn_stats", "bdl_launch_count",
    "bdl_profile", "bdl_profile_read", "bdl_kernel_count", "bdl_kernel_name", "bdl_knn_noalloc",
    "bdl_insert_batch", "bdl_erase_batch", "bdl_knn_batch",
    "bdl_server_default_config", "bdl_server_create", "bdl_server_submit", "bdl_server_wait",
    "bdl_server_drain", "bdl_server_stats", "bdl_server_destroy", "bdl_server_now_ms",
    "bdl_knn_plan_create", "bdl_knn_plan_launch", "bdl_knn_plan_destroy", "bdl_next_id",
    "bdl_knn_count", "bdl_poll_error", "bdl_profile_read_bytes", "bdl_profile_timeline", "bdl_set_knn_shape",
]

BDL_REQ_INSERT, BDL_REQ_ERASE, BDL_REQ_KNN = 0, 1, 2


class BdlConfig(ctypes.Structure):
    _fields_ = [("leaf_size", ctypes.c_int32), ("buffer_size", ctypes.c_int32),
                ("bloom_bits_per_key", ctypes.c_int32), ("bloom_hashes", ctypes.c_int32),
                ("hash_seed", ctypes.c_uint64), ("hbm_budget_bytes", ctypes.c_int64),
                ("split_rule", ctypes.c_int32), ("reserved_", ctypes.c_int32)]


BDL_SPLIT_OBJECT, BDL_SPLIT_SPATIAL = 0, 1


class BdlRequest(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("k", ctypes.c_int32), ("n", ctypes.c_int64),
                ("in_host", ctypes.c_void_p), ("out_ids_host", ctypes.c_void_p),
                ("out_d2_host", ctypes.c_void_p)]


class BdlResult(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("kind", ctypes.c_int32), ("done", ctypes.c_int32),
                ("pad_", ctypes.c_int32), ("ticket", ctypes.c_uint64), ("n_done", ctypes.c_int64),
                ("group", ctypes.c_int64), ("t_submit_ms", ctypes.c_double),
                ("t_start_ms", ctypes.c_double), ("t_done_ms", ctypes.c_double)]


class BdlServerConfig(ctypes.Structure):
    _fields_ = [("max_inflight", ctypes.c_int32), ("serial", ctypes.c_int32),
                ("staging_budget_bytes", ctypes.c_int64), ("max_group_queries", ctypes.c_int64),
                ("max_group_points", ctypes.c_int64)]


class BdlError(RuntimeError):
    def __init__(self, status, where, msg):
        super().__init__("%s failed: status %d (%s): %s" % (where, status, status_string(status), msg))
        self.status = status


_lib = None


def load(path=None):
    """Load the shared library (build it first with build_lib.build())."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError("CUDA library not built: %s is missing (run __graft_entry__.build())" % path)
    L = ctypes.CDLL(path)
    P, i32, i64, u64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_uint64
    sig = {
        "bdl_default_config": (None, [P]),
        "bdl_create": (i32, [i32, P, P, i64, P, P, P]),
        "bdl_insert": (i32, [P, P, i64, P, P]),
        "bdl_erase": (i32, [P, P, i64, P, P]),
        "bdl_knn": (i32, [P, P, i64, i32, P, P, P]),
        "bdl_size": (i32, [P, P]),
        "bdl_destroy": (i32, [P]),
        "bdl_status_string": (ctypes.c_char_p, [i32]),
        "bdl_last_error": (ctypes.c_char_p, []),
        "bdl_tree_mask": (i32, [P, P, P]),
        "bdl_buffer_ids": (i32, [P, P, i64, P, P]),
        "bdl_tree_info": (i32, [P, i32, P]),
        "bdl_tree_export": (i32, [P, i32, P, P, P, P, P, P, P]),
        "bdl_bloom_export": (i32, [P, i32, P, P]),
        "bdl_knn_stats": (i32, [P, i32, P]),
        "bdl_launch_count": (u64, []),
        "bdl_profile": (i32, [i32]),
        "bdl_profile_read": (i32, [P, P, i32]),
        "bdl_kernel_count": (i32, []),
        "bdl_kernel_name": (ctypes.c_char_p, [i32]),
        "bdl_knn_noalloc": (i32, [P, P, i64, i32, P, P, P]),
        "bdl_insert_batch": (i32, [P, i32, P, P, P, P]),
        "bdl_erase_batch": (i32, [P, i32, P, P, P, P]),
        "bdl_knn_batch": (i32, [P, i32, P, P, i32, P, P, P]),
        "bdl_server_default_config": (None, [P]),
        "bdl_server_create": (i32, [P, P, P]),
        "bdl_server_submit": (i32, [P, P, P]),
        "bdl_server_wait": (i32, [P, u64, P]),
        "bdl_server_drain": (i32, [P]),
        "bdl_server_stats": (i32, [P, P]),
        "bdl_server_destroy": (i32, [P]),
        "bdl_server_now_ms": (ctypes.c_double, [P]),
        "bdl_knn_plan_create": (i32, [P, i32, P, P, i32, P, P, P, P]),
        "bdl_knn_plan_launch": (i32, [P, P]),
        "bdl_knn_plan_destroy": (i32, [P]),
        "bdl_next_id": (i32, [P, P]),
        "bdl_knn_count": (i32, [P, P, i64, i32, P, P, P, P]),
        "bdl_poll_error": (i32, [P, P, P]),
        "bdl_set_knn_shape": (i32, [P, i32, i32]),
        "bdl_profile_read_bytes": (i32, [P, P, P, i32]),
        "bdl_profile_timeline": (i32, [P, P, P, P, i32, P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def status_string(st):
    return load().bdl_status_string(st).decode()


def last_error():
    return load().bdl_last_error().decode()


def check(st, where):
    if st != BDL_OK:
        raise BdlError(st, where, last_error())
    return st


def _ref(x):
    return ctypes.byref(x)


# --- entry points (same names as the C ABI) --------------------------------

def bdl_default_config():
    cfg = BdlConfig()
    load().bdl_default_config(_ref(cfg))
    return cfg


def bdl_create(dim, cfg, pts_dev, n, out_ids_dev, stream):
    """Returns (status, forest handle)."""
    h = ctypes.c_void_p()
    st = load().bdl_create(dim, _ref(cfg) if cfg is not None else None, pts_dev, n,
                           out_ids_dev, stream, _ref(h))
    return st, h.value


def bdl_insert(f, pts_dev, n, out_ids_dev, stream):
    return load().bdl_insert(f, pts_dev, n, out_ids_dev, stream)


def bdl_erase(f, ids_dev, n, stream):
    """Returns (status, number erased)."""
    out = ctypes.c_int64(0)
    st = load().bdl_erase(f, ids_dev, n, _ref(out), stream)
    return st, out.value


def bdl_knn(f, q_dev, m, k, out_ids_dev, out_d2_dev, stream):
    return load().bdl_knn(f, q_dev, m, k, out_ids_dev, out_d2_dev, stream)


def bdl_knn_count(f, q_dev, m, k, out_ids_dev, out_d2_dev, counts_dev, stream):
    """bdl_knn by the counting instance: adds (nodes, points, queries) into the
    device array counts_dev[3] (uint64)."""
    return load().bdl_knn_count(f, q_dev, m, k, out_ids_dev, out_d2_dev, counts_dev, stream)


def bdl_poll_error(f, stream):
    """Returns (status, device error word bits); waits for the stream."""
    bits = ctypes.c_uint64(0)
    st = load().bdl_poll_error(f, _ref(bits), stream)
    return st, bits.value


def bdl_set_knn_shape(f, block_threads, queries_per_warp):
    """Launch shape of the forest's k-NN kernel (block size, queries per warp)."""
    return load().bdl_set_knn_shape(f, block_threads, queries_per_warp)


def bdl_knn_noalloc(f, q_dev, m, k, out_ids_dev, out_d2_dev, stream):
    """bdl_knn without device allocation (scratch in a fixed library array)."""
    return load().bdl_knn_noalloc(f, q_dev, m, k, out_ids_dev, out_d2_dev, stream)


def _ptr_array(xs):
    return (ctypes.c_void_p * max(len(xs), 1))(*[x or None for x in xs])


def _i64_array(xs):
    return (ctypes.c_int64 * max(len(xs), 1))(*xs)


def bdl_insert_batch(forests, pts_dev, n, out_ids_dev, stream):
    """Insert_L on len(forests) forests; lists of handles / device pointers / sizes."""
    return load().bdl_insert_batch(_ptr_array(forests), len(forests), _ptr_array(pts_dev),
                                   _i64_array(n), _ptr_array(out_ids_dev), stream)


def bdl_erase_batch(forests, ids_dev, n, stream):
    """Returns (status, [number erased per forest])."""
    out = (ctypes.c_int64 * max(len(forests), 1))()
    st = load().bdl_erase_batch(_ptr_array(forests), len(forests), _ptr_array(ids_dev),
                                _i64_array(n), out, stream)
    return st, [int(out[i]) for i in range(len(forests))]


def bdl_knn_batch(forests, q_dev, m, k, out_ids_dev, out_d2_dev, stream):
    return load().bdl_knn_batch(_ptr_array(forests), len(forests), _ptr_array(q_dev), _i64_array(m),
                                k, _ptr_array(out_ids_dev), _ptr_array(out_d2_dev), stream)


def bdl_knn_plan_create(forests, q_dev, m, k, out_ids_dev, out_d2_dev, stream):
    """Returns (status, plan handle)."""
    h = ctypes.c_void_p()
    st = load().bdl_knn_plan_create(_ptr_array(forests), len(forests), _ptr_array(q_dev), _i64_array(m), k,
                                    _ptr_array(out_ids_dev), _ptr_array(out_d2_dev), stream, _ref(h))
    return st, h.value


def bdl_knn_plan_launch(plan, stream):
    return load().bdl_knn_plan_launch(plan, stream)


def bdl_knn_plan_destroy(plan):
    return load().bdl_knn_plan_destroy(plan)


def bdl_server_default_config():
    cfg = BdlServerConfig()
    load().bdl_server_default_config(_ref(cfg))
    return cfg


def bdl_server_create(f, cfg):
    """Returns (status, server handle)."""
    h = ctypes.c_void_p()
    st = load().bdl_server_create(f, _ref(cfg) if cfg is not None else None, _ref(h))
    return st, h.value


def bdl_server_submit(s, req):
    """Returns (status, ticket)."""
    t = ctypes.c_uint64(0)
    st = load().bdl_server_submit(s, _ref(req), _ref(t))
    return st, t.value


def bdl_server_wait(s, ticket):
    """Returns (status, BdlResult)."""
    r = BdlResult()
    st = load().bdl_server_wait(s, ticket, _ref(r))
    return st, r


def bdl_server_drain(s):
    return load().bdl_server_drain(s)


def bdl_server_stats(s):
    g = ctypes.c_int64(0)
    st = load().bdl_server_stats(s, _ref(g))
    return st, g.value


def bdl_server_now_ms(s):
    return float(load().bdl_server_now_ms(s))


def bdl_server_destroy(s):
    return load().bdl_server_destroy(s)


def bdl_size(f):
    out = ctypes.c_int64(0)
    st = load().bdl_size(f, _ref(out))
    return st, out.value


def bdl_next_id(f):
    out = ctypes.c_int64(0)
    st = load().bdl_next_id(f, _ref(out))
    return st, out.value


def bdl_destroy(f):
    return load().bdl_destroy(f)


def bdl_tree_mask(f):
    m = ctypes.c_uint64(0)
    nb = ctypes.c_int64(0)
    st = load().bdl_tree_mask(f, _ref(m), _ref(nb))
    return st, m.value, nb.value


def bdl_buffer_ids(f, out_host_ptr, cap, stream):
    n = ctypes.c_int64(0)
    st = load().bdl_buffer_ids(f, out_host_ptr, cap, _ref(n), stream)
    return st, n.value


def bdl_tree_info(f, level, info_host_ptr):
    return load().bdl_tree_info(f, level, info_host_ptr)


def bdl_tree_export(f, level, key, child, box, live, leaf_off, ids, stream):
    return load().bdl_tree_export(f, level, key, child, box, live, leaf_off, ids, stream)


def bdl_bloom_export(f, level, words, stream):
    return load().bdl_bloom_export(f, level, words, stream)


def bdl_knn_stats(f, enable, out_host_ptr):
    return load().bdl_knn_stats(f, enable, out_host_ptr)


def bdl_launch_count():
    return int(load().bdl_launch_count())


def bdl_profile(enable):
    return load().bdl_profile(1 if enable else 0)


def bdl_profile_read():
    """{kernel name: (total ms, launches)} since the last read (waits for the events)."""
    n = load().bdl_kernel_count()
    ms = (ctypes.c_double * n)()
    cnt = (ctypes.c_int64 * n)()
    check(load().bdl_profile_read(ms, cnt, n), "bdl_profile_read")
    return {bdl_kernel_name(i): (ms[i], cnt[i]) for i in range(n) if cnt[i]}


def bdl_profile_read_bytes():
    """{kernel name: (total ms, launches, algorithmic bytes)} since the last read."""
    n = load().bdl_kernel_count()
    ms = (ctypes.c_double * n)()
    cnt = (ctypes.c_int64 * n)()
    by = (ctypes.c_double * n)()
    check(load().bdl_profile_read_bytes(ms, cnt, by, n), "bdl_profile_read_bytes")
    return {bdl_kernel_name(i): (ms[i], cnt[i], by[i]) for i in range(n) if cnt[i]}


def bdl_profile_timeline(cap=1 << 16):
    """[(kernel name, start ms, end ms, algorithmic bytes)] of the recorded
    launches in launch order (does not clear the records)."""
    kid = (ctypes.c_int32 * cap)()
    a = (ctypes.c_double * cap)()
    b = (ctypes.c_double * cap)()
    by = (ctypes.c_double * cap)()
    n = ctypes.c_int(0)
    check(load().bdl_profile_timeline(kid, a, b, by, cap, _ref(n)), "bdl_profile_timeline")
    return [(bdl_kernel_name(kid[i]), a[i], b[i], by[i]) for i in range(min(cap, n.value))]


def bdl_kernel_count():
    return int(load().bdl_kernel_count())


def bdl_kernel_name(i):
    return load().bdl_kernel_name(i).decode()
