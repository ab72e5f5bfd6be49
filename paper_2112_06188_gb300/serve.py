"""Python handle on the request server of the C ABI (bdl_server_*): argument
marshalling only -- admission, batching, execution and completion all run in
the library's own threads and CUDA streams.

Host buffers handed to a request must stay alive until it is collected; this
wrapper keeps them referenced.  Pinned tensors let the copies overlap with
the device work of other requests.
"""
import numpy as np
import torch

from . import capi


def _pinned(x, dtype):
    if isinstance(x, np.ndarray):
        x = torch.from_numpy(np.ascontiguousarray(x))
    x = torch.as_tensor(x).to(dtype).contiguous()
    if x.is_cuda:
        raise ValueError("request buffers live in host memory")
    return x if x.is_pinned() else x.pin_memory()


class Server:
    """Continuous-batching request server on one resident Forest."""

    def __init__(self, forest, max_inflight=64, serial=False, staging_budget_bytes=1 << 30,
                 max_group_queries=1 << 20, max_group_points=1 << 21):
        self.forest = forest
        cfg = capi.bdl_server_default_config()
        cfg.max_inflight, cfg.serial = max_inflight, 1 if serial else 0
        cfg.staging_budget_bytes = staging_budget_bytes
        cfg.max_group_queries, cfg.max_group_points = max_group_queries, max_group_points
        st, h = capi.bdl_server_create(forest._h, cfg)
        capi.check(st, "bdl_server_create")
        self._h = h
        self._keep = {}

    def _submit(self, kind, data, k=0, out_ids=None, out_d2=None, n=None):
        req = capi.BdlRequest()
        req.kind, req.k = kind, k
        req.n = n
        req.in_host = data.data_ptr() if data.numel() else None
        req.out_ids_host = out_ids.data_ptr() if out_ids is not None and out_ids.numel() else None
        req.out_d2_host = out_d2.data_ptr() if out_d2 is not None and out_d2.numel() else None
        st, t = capi.bdl_server_submit(self._h, req)
        capi.check(st, "bdl_server_submit")
        self._keep[t] = (kind, data, out_ids, out_d2)
        return t

    def insert(self, points, out=None):
        """Queue Insert_L of `points`; `out` (pinned int32 [n]) receives the ids."""
        p = _pinned(points, torch.int32).reshape(-1, self.forest.dim)
        ids = out if out is not None else torch.empty(p.shape[0], dtype=torch.int32).pin_memory()
        return self._submit(capi.BDL_REQ_INSERT, p, out_ids=ids, n=p.shape[0])

    def erase(self, ids):
        i = _pinned(ids, torch.int32).reshape(-1)
        return self._submit(capi.BDL_REQ_ERASE, i, n=i.shape[0])

    def knn(self, queries, k, out=None):
        """Queue kNN_L; `out` = (pinned int32 [m, k], pinned int64 [m, k]) receives the rows."""
        q = _pinned(queries, torch.int32).reshape(-1, self.forest.dim)
        if out is None:
            oi = torch.empty((q.shape[0], k), dtype=torch.int32).pin_memory()
            od = torch.empty((q.shape[0], k), dtype=torch.int64).pin_memory()
        else:
            oi, od = out
        return self._submit(capi.BDL_REQ_KNN, q, k=k, out_ids=oi, out_d2=od, n=q.shape[0])

    def wait(self, ticket):
        """The request's result: a dict with status, n_done, timestamps (ms) and
        its outputs (insert: ids; k-NN: ids, d2)."""
        st, r = capi.bdl_server_wait(self._h, ticket)
        capi.check(st, "bdl_server_wait")
        kind, data, oi, od = self._keep.pop(ticket)
        out = {"status": r.status, "kind": r.kind, "n_done": r.n_done, "group": r.group,
               "t_submit_ms": r.t_submit_ms, "t_start_ms": r.t_start_ms, "t_done_ms": r.t_done_ms}
        if kind == capi.BDL_REQ_INSERT:
            out["ids"] = oi
        elif kind == capi.BDL_REQ_KNN:
            out["ids"], out["d2"] = oi, od
        return out

    def drain(self):
        capi.check(capi.bdl_server_drain(self._h), "bdl_server_drain")

    def now_ms(self):
        """The server's clock (ms since creation), the clock of the results' timestamps."""
        return capi.bdl_server_now_ms(self._h)

    def groups(self):
        st, g = capi.bdl_server_stats(self._h)
        capi.check(st, "bdl_server_stats")
        return g

    def close(self):
        if getattr(self, "_h", None):
            capi.bdl_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
