"""Pythonic wrapper over the C ABI: a Forest object taking torch tensors.

Device tensors are passed straight through; host tensors are copied to the
device on the forest's stream and results copied back (the end-to-end path).
PyTorch only provides memory and streams here -- every step of the method
runs in the CUDA library.
"""
import ctypes

import numpy as np
import torch

from . import capi


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None and t.numel() else None


def _addr(t):
    return t.data_ptr() if t is not None and t.numel() else None


def _stream_handle(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


GRID = 1 << 20                      # coordinates lie in [0, 2^20)
I32_MIN, I32_MAX = -(1 << 31), (1 << 31) - 1


def _int_tensor(x):
    """x as a torch tensor of an integer dtype (numpy arrays, lists and tensors
    accepted; floating-point or boolean data is refused rather than rounded)."""
    if isinstance(x, np.ndarray):
        x = torch.from_numpy(np.ascontiguousarray(x))
    x = torch.as_tensor(x)
    if x.dtype.is_floating_point or x.dtype.is_complex or x.dtype == torch.bool:
        raise TypeError("integer data expected, got %s" % x.dtype)
    return x


def _narrow_i32(x, lo, hi, what):
    """x cast to int32, after checking (when the cast would narrow) that every
    value lies in [lo, hi]: a wider value must not wrap onto another one."""
    if x.dtype == torch.int32:
        return x
    if x.numel():
        mn, mx = (int(v) for v in torch.aminmax(x))
        if mn < lo or mx > hi:
            raise ValueError("%s outside [%d, %d] (got %d .. %d)" % (what, lo, hi, mn, mx))
    return x.to(torch.int32)


def _coords_i32(x):
    return _narrow_i32(_int_tensor(x), 0, GRID - 1, "coordinates")


def _ids_i32(x):
    return _narrow_i32(_int_tensor(x), I32_MIN, I32_MAX, "ids")


class Forest:
    """A batch-dynamic kd-tree forest resident on one GPU."""

    def __init__(self, dim, points=None, leaf_size=16, buffer_size=1024, bloom_bits_per_key=16,
                 hash_seed=0x5EED, hbm_budget_bytes=0, device=None, stream=None, split="object"):
        """split: "object" (median point, Alg. 1) or "spatial" (midpoint of the
        extent, Sec. V-C); k-NN answers are the same either way."""
        capi.load()
        self.dim = dim
        dev = torch.device(device or "cuda")
        if dev.type == "cuda" and dev.index is None:   # "cuda": the current device, by index
            dev = torch.device("cuda", torch.cuda.current_device())
        self.device = dev
        self.stream = stream
        cfg = capi.bdl_default_config()
        cfg.leaf_size, cfg.buffer_size = leaf_size, buffer_size
        cfg.bloom_bits_per_key, cfg.hash_seed = bloom_bits_per_key, hash_seed
        cfg.hbm_budget_bytes = hbm_budget_bytes
        if split not in ("object", "spatial"):
            raise ValueError("split must be 'object' or 'spatial'")
        cfg.split_rule = capi.BDL_SPLIT_SPATIAL if split == "spatial" else capi.BDL_SPLIT_OBJECT
        self.split = split
        self.cfg = cfg
        with torch.cuda.device(self.device):
            st, h = capi.bdl_create(dim, cfg, None, 0, None, _stream_handle(stream))
        capi.check(st, "bdl_create")
        self._h = h
        if points is not None:
            self.insert(points)

    def close(self):
        if getattr(self, "_h", None):
            capi.bdl_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _stream(self):
        return self.stream if self.stream is not None else torch.cuda.current_stream(self.device)

    def _dev(self, x):
        """Contiguous int32 tensor of x (already narrowed) on the forest's
        device; host data goes through pinned memory on the forest's stream,
        a tensor on another GPU is copied over."""
        if x.is_cuda:
            if x.device != self.device:
                x = x.to(self.device)
            return x.contiguous()
        x = x.contiguous()
        if not x.is_pinned():
            x = x.pin_memory()
        with torch.cuda.stream(self._stream()):
            return x.to(self.device, non_blocking=True)

    def _host(self, t):
        self._stream().synchronize()
        return t.cpu()

    def insert(self, points):
        """Insert_L: returns the new ids (device tensor if points were on the
        device; for host points a host tensor, known without a device read:
        the ids are consecutive)."""
        on_host = not (isinstance(points, torch.Tensor) and points.is_cuda)
        p = self._dev(_coords_i32(points)).reshape(-1, self.dim)
        if on_host:
            capi.check(capi.bdl_insert(self._h, _ptr(p), p.shape[0], None, _stream_handle(self.stream)),
                       "bdl_insert")
            st, nxt = capi.bdl_next_id(self._h)
            capi.check(st, "bdl_next_id")
            return torch.arange(nxt - p.shape[0], nxt, dtype=torch.int32)
        ids = torch.empty(p.shape[0], dtype=torch.int32, device=self.device)
        capi.check(capi.bdl_insert(self._h, _ptr(p), p.shape[0], _ptr(ids),
                                   _stream_handle(self.stream)), "bdl_insert")
        return ids

    def erase(self, ids):
        """Erase_L: returns the number of points erased."""
        i = self._dev(_ids_i32(ids)).reshape(-1)
        st, n = capi.bdl_erase(self._h, _ptr(i), i.shape[0], _stream_handle(self.stream))
        capi.check(st, "bdl_erase")
        return n

    def knn(self, queries, k, out=None):
        """kNN_L: (ids [m,k] int32, d2 [m,k] int64), sorted by (d2, id)."""
        on_host = not (isinstance(queries, torch.Tensor) and queries.is_cuda)
        q = self._dev(_coords_i32(queries)).reshape(-1, self.dim)
        m = q.shape[0]
        if out is None:
            oi = torch.empty((m, k), dtype=torch.int32, device=self.device)
            od = torch.empty((m, k), dtype=torch.int64, device=self.device)
        else:
            oi, od = out
            _check_out(oi, od, m, k, self.device)
        capi.check(capi.bdl_knn(self._h, _ptr(q), m, k, _ptr(oi), _ptr(od),
                                _stream_handle(self.stream)), "bdl_knn")
        if on_host:
            return self._host(oi), self._host(od)
        return oi, od

    def size(self):
        st, n = capi.bdl_size(self._h)
        capi.check(st, "bdl_size")
        return n

    def tree_mask(self):
        st, m, nb = capi.bdl_tree_mask(self._h)
        capi.check(st, "bdl_tree_mask")
        return m

    def tree_levels(self):
        m = self.tree_mask()
        return [i for i in range(64) if (m >> i) & 1]

    def buffer_ids(self):
        out = np.empty(self.cfg.buffer_size, dtype=np.int32)
        st, n = capi.bdl_buffer_ids(self._h, out.ctypes.data_as(ctypes.c_void_p), len(out),
                                    _stream_handle(self.stream))
        capi.check(st, "bdl_buffer_ids")
        return out[:n].copy()

    def tree(self, level):
        """Tree `level` as numpy arrays, in the layout the oracle exports."""
        info = np.zeros(6, dtype=np.int64)
        if capi.bdl_tree_info(self._h, level, info.ctypes.data_as(ctypes.c_void_p)) != 0:
            return None
        size, live, h, nn, blocks = (int(x) for x in info[:5])
        d = self.dim
        key = np.empty(nn, np.int64)
        child = np.empty(2 * nn, np.int32)
        box = np.empty(nn * 2 * d, np.int32)
        nlive = np.empty(nn, np.int32)
        leaf_off = np.empty((1 << h) + 1, np.int32)
        ids = np.empty(size, np.int32)
        P = lambda a: a.ctypes.data_as(ctypes.c_void_p)
        capi.check(capi.bdl_tree_export(self._h, level, P(key), P(child), P(box), P(nlive),
                                        P(leaf_off), P(ids), _stream_handle(self.stream)),
                   "bdl_tree_export")
        bloom = None
        if blocks:
            bloom = np.empty(blocks * 8, np.uint32)
            capi.check(capi.bdl_bloom_export(self._h, level, P(bloom), _stream_handle(self.stream)),
                       "bdl_bloom_export")
        dead = ids < 0
        real = np.where(dead, ids & 0x7FFFFFFF, ids).astype(np.int32)
        return dict(size=size, live=live, h=h, nnodes=nn, key=key, child=child.reshape(nn, 2),
                    box=box.reshape(nn, 2 * d), node_live=nlive, leaf_off=leaf_off,
                    ids=real, dead=dead, bloom=bloom)

    def knn_count(self, queries, k, counts, out=None):
        """kNN_L through the counting instance (same rows); adds the nodes
        visited, live leaf points examined and queries to `counts`, a (3,)
        int64 device tensor the caller zeroes.  Measurement only."""
        q = self._dev(_coords_i32(queries)).reshape(-1, self.dim)
        m = q.shape[0]
        if out is None:
            out = (torch.empty((m, k), dtype=torch.int32, device=self.device),
                   torch.empty((m, k), dtype=torch.int64, device=self.device))
        _check_out(out[0], out[1], m, k, self.device)
        if counts.dtype != torch.int64 or counts.numel() != 3 or counts.device != self.device:
            raise ValueError("counts must be a (3,) int64 tensor on the forest's device")
        capi.check(capi.bdl_knn_count(self._h, _ptr(q), m, k, _ptr(out[0]), _ptr(out[1]), _ptr(counts),
                                      _stream_handle(self.stream)), "bdl_knn_count")
        return out

    def poll_error(self):
        """The device error word (0 when no kernel found an index outside its
        buffers); waits for the forest's stream."""
        st, bits = capi.bdl_poll_error(self._h, _stream_handle(self.stream))
        if st not in (capi.BDL_OK, capi.BDL_EINTERNAL):
            capi.check(st, "bdl_poll_error")
        return bits

    def set_knn_shape(self, block_threads=128, queries_per_warp=32):
        """Launch shape of this forest's k-NN kernel: threads per block (64,
        128, 256) and queries per warp (32, 64, 128).  Results do not depend
        on it."""
        capi.check(capi.bdl_set_knn_shape(self._h, int(block_threads), int(queries_per_warp)),
                   "bdl_set_knn_shape")

    def knn_stats(self, enable=None):
        """enable=True/False switches per-query visit counting on/off (and resets);
        enable=None reads (nodes visited, leaf points examined, queries)."""
        if enable is None:
            out = np.zeros(3, np.int64)
            capi.check(capi.bdl_knn_stats(self._h, 0, out.ctypes.data_as(ctypes.c_void_p)),
                       "bdl_knn_stats")
            return tuple(int(x) for x in out)
        capi.check(capi.bdl_knn_stats(self._h, 1 if enable else 0, None), "bdl_knn_stats")
        return None


def _check_out(oi, od, m, k, device):
    """The caller's output buffers of a k-NN call: contiguous (m, k) int32 ids
    and int64 squared distances on the forest's device (the kernel writes
    m * k entries of each)."""
    for t, dt, name in ((oi, torch.int32, "ids"), (od, torch.int64, "d2")):
        if not isinstance(t, torch.Tensor):
            raise TypeError("out %s must be a tensor" % name)
        if t.dtype != dt or tuple(t.shape) != (m, k) or not t.is_contiguous():
            raise ValueError("out %s must be a contiguous (%d, %d) %s tensor, got %s %s" %
                             (name, m, k, dt, tuple(t.shape), t.dtype))
        if not t.is_cuda or t.device != torch.device(device):
            raise ValueError("out %s must be on %s, not %s" % (name, device, t.device))


# --- batched forests: one call for many independent forests -----------------

def _batch_stream(forests, stream):
    if stream is None and forests:
        stream = forests[0]._stream()
    return _stream_handle(stream)


def insert_batch(forests, points, stream=None):
    """Insert_L on every forest; points[i] is a device tensor [n_i, dim_i].
    Returns the list of id tensors."""
    ps = [f._dev(_coords_i32(p)).reshape(-1, f.dim) for f, p in zip(forests, points)]
    ids = [torch.empty(p.shape[0], dtype=torch.int32, device=p.device) for p in ps]
    capi.check(capi.bdl_insert_batch([f._h for f in forests], [_addr(p) for p in ps],
                                     [p.shape[0] for p in ps], [_addr(i) for i in ids],
                                     _batch_stream(forests, stream)), "bdl_insert_batch")
    return ids


def erase_batch(forests, ids, stream=None):
    """Erase_L on every forest; returns the list of counts erased."""
    ts = [f._dev(_ids_i32(i)).reshape(-1) for f, i in zip(forests, ids)]
    st, n = capi.bdl_erase_batch([f._h for f in forests], [_addr(t) for t in ts],
                                 [t.shape[0] for t in ts], _batch_stream(forests, stream))
    capi.check(st, "bdl_erase_batch")
    return n


def knn_batch(forests, queries, k, out=None, stream=None):
    """kNN_L on every forest; queries[i] is a device tensor [m_i, dim_i].
    Returns a list of (ids [m_i, k], d2 [m_i, k])."""
    qs = [f._dev(_coords_i32(q)).reshape(-1, f.dim) for f, q in zip(forests, queries)]
    if out is None:
        out = [(torch.empty((q.shape[0], k), dtype=torch.int32, device=q.device),
                torch.empty((q.shape[0], k), dtype=torch.int64, device=q.device)) for q in qs]
    else:
        for f, q, (oi, od) in zip(forests, qs, out):
            _check_out(oi, od, q.shape[0], k, f.device)
    capi.check(capi.bdl_knn_batch([f._h for f in forests], [_addr(q) for q in qs],
                                  [q.shape[0] for q in qs], k, [_addr(o[0]) for o in out],
                                  [_addr(o[1]) for o in out], _batch_stream(forests, stream)),
               "bdl_knn_batch")
    return out


class KnnPlan:
    """A prepared kNN_L over forests[i] with the device query tensors queries[i]:
    launch() answers whatever the query tensors hold at that time (same
    shapes), against the forests as they were when the plan was made.  A launch
    issues kernels only, so it can be captured in a CUDA graph."""

    def __init__(self, forests, queries, k, out=None, stream=None):
        self.queries = [q.reshape(-1, f.dim) for f, q in zip(forests, queries)]
        for q in self.queries:
            if q.dtype != torch.int32 or not q.is_contiguous() or not q.is_cuda:
                raise ValueError("plan queries must be contiguous int32 device tensors")
        if out is None:
            out = [(torch.empty((q.shape[0], k), dtype=torch.int32, device=q.device),
                    torch.empty((q.shape[0], k), dtype=torch.int64, device=q.device)) for q in self.queries]
        else:
            for f, q, (oi, od) in zip(forests, self.queries, out):
                _check_out(oi, od, q.shape[0], k, f.device)
        self.out = out
        self.forests = list(forests)
        st, h = capi.bdl_knn_plan_create([f._h for f in forests], [_addr(q) for q in self.queries],
                                         [q.shape[0] for q in self.queries], k, [_addr(o[0]) for o in out],
                                         [_addr(o[1]) for o in out], _batch_stream(forests, stream))
        capi.check(st, "bdl_knn_plan_create")
        self._h = h

    def launch(self, stream=None):
        capi.check(capi.bdl_knn_plan_launch(self._h, _batch_stream(self.forests, stream)), "bdl_knn_plan_launch")
        return self.out

    def close(self):
        if getattr(self, "_h", None):
            capi.bdl_knn_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
