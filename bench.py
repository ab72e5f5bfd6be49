"""Benchmark of the BDL-tree hot path on one GB300 (or N, one forest per GPU).

Workload (3-D uniform int32 points on the 2^20 grid, leaf size 16, X = 1024):
a forest of 10M points is built once; one step is then the whole hot path on
one batch -- insert 1M new points (Insert_L), erase 1M ids drawn uniformly
from the live set (Erase_L), and answer k = 10 nearest neighbours for 1M
queries drawn from the live set (kNN_L).  The forest stays at ~10M points.

Metric: operations per second of the step -- (points inserted + points
erased + queries answered) / step time -- with updates/s and queries/s of the
two phases beside it.  Inputs are resident in HBM before the timed region;
L2 is flushed (256 MB write) between steps, outside the timed events.

--impl reference times the CPU oracle (oracle/) as it stands on the host
cores, on a 1/10-scale sample of the same step.

--workload forests runs the batched-forests workload instead: 512
independent 2-D/3-D forests of log-uniform sizes in [1k, 200k]; one step gives
every forest an insert batch of 5-20% of its size, a delete batch of 2-10% of
its live ids and k = 8 queries (1-5k per forest).  The step runs once through
the batched entry points (one call per operation for all forests) and once
as per-forest calls on an identical second set of forests; both results must
be identical, and both times are reported.

--workload serve runs the serving workload: one resident 5-D forest growing
from 1M to 50M points under a Poisson stream of insert (1k-1M points), erase
(1k-500k live ids) and k-NN (1-100k queries, k in {1, 5, 10}) requests in a
4:1:5 mix, served by the library's continuous-batching server under a fixed
device-memory budget, and again by its one-request-at-a-time mode; p50/p99
latency per request type and sustained updates/s and queries/s are reported.

--workload sweep runs the paper's sweeps (Sec. VI) on two 10M-point sets, a 2-D
Gaussian-cluster mixture (standing in for the 2-D VisualVar set) and 7-D
uniform points: insert throughput against the batch size when the whole set is
inserted batch by batch into an empty forest, erase throughput against the
batch size when the whole set is erased batch by batch, and k-NN throughput
(every point queried: the k-NN graph) against k = 2..11 after the set was
inserted in 5% batches.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "batch updates/sec and k-NN queries/sec at 10M pts; HBM GB/s; serve p50/p99 ms"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n0", type=int, default=10_000_000)
    ap.add_argument("--batch", type=int, default=1_000_000)
    ap.add_argument("--queries", type=int, default=1_000_000)
    ap.add_argument("--k", type=int, default=None, help="default 10 (forest10m), 8 (forests)")
    ap.add_argument("--dim", type=int, default=3)
    ap.add_argument("--leaf", default="auto",
                    help="leaf size, or 'auto': autotuned in {8, 12, 16, 24, 32} on this workload before timing")
    ap.add_argument("--knn-shape", default="128x32",
                    help="k-NN launch shape BLOCKxQUERIES_PER_WARP (64/128/256 x 32/64/128) when --leaf "
                         "is given; with --leaf auto the autotuner picks it after the leaf size")
    ap.add_argument("--e2e-steps", type=int, default=None,
                    help="end-to-end steps after the timed ones (default: as many as --steps)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="forest10m", choices=["forest10m", "forests", "serve", "sweep"])
    ap.add_argument("--split", default="object", choices=["object", "spatial"],
                    help="splitting rule of the trees (Sec. V-C)")
    ap.add_argument("--rate", type=float, default=600.0, help="serve: requests per second")
    ap.add_argument("--n-final", type=int, default=50_000_000, help="serve: stop at this many points")
    ap.add_argument("--forests", type=int, default=512)
    a = ap.parse_args()
    if a.k is None:
        a.k = 8 if a.workload == "forests" else 10
    if a.e2e_steps is None:
        a.e2e_steps = a.steps
    return a


def parse_shape(text):
    """'BLOCKxQPW' -> (block threads, queries per warp)."""
    b, q = text.lower().split("x")
    return int(b), int(q)


def shape_record(shape, ms_by_shape, seconds, inputs_text):
    """The autotune record of the k-NN launch shape."""
    return {"candidates_ms_per_knn": {"%dx%d" % sh: round(v, 3) for sh, v in ms_by_shape.items()},
            "chosen": {"block_threads": shape[0], "queries_per_warp": shape[1]},
            "tuning_s": round(seconds, 2), "inputs": inputs_text}


def workload_config(a, n_gpus):
    return {"workload": "3-D uniform int32 forest of %d points; per step insert %d, erase %d "
                        "live ids, k=%d NN for %d live-set queries" % (a.n0, a.batch, a.batch, a.k, a.queries),
            "dim": a.dim, "n0": a.n0, "insert_batch": a.batch, "erase_batch": a.batch,
            "queries": a.queries, "k": a.k, "leaf_size": a.leaf, "knn_shape": a.knn_shape,
            "buffer_size": 1024, "split": a.split,
            "l2": "flushed between steps (256 MB write), inputs resident in HBM",
            "parallelism": "one independent forest per GPU" if n_gpus > 1 else "single GPU"}


# ---------------------------------------------------------------------------
# inputs (shared by both arms)
# ---------------------------------------------------------------------------

class StepInputs:
    """Pre-drawn inputs of consecutive steps on a forest of n0 points."""

    def __init__(self, n0, batch, queries, dim, nsteps, seed):
        from paper_2112_06188_gb300 import inputs
        self.initial = inputs.uniform_points(n0, dim, seed)
        live = inputs.LiveSet(dim)
        live.insert(self.initial)
        rng = np.random.default_rng(seed + 1000)
        self.steps = []
        for s in range(nsteps):
            ins = rng.integers(0, inputs.GRID, size=(batch, dim), dtype=np.int32)
            live.insert(ins)
            ids = live.live_ids()
            era = rng.choice(ids, size=min(batch, len(ids)), replace=False).astype(np.int32)
            live.erase(era)
            lid = live.live_ids()
            q = live.coords[lid[rng.integers(0, len(lid), size=queries)]]
            self.steps.append((ins, era, np.ascontiguousarray(q)))


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), "bdl_clocks_%d.csv" % os.getpid())

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], [], set()
        names = ["active", "hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            for line in fh:
                p = [x.strip() for x in line.split(",")]
                if len(p) < 9:
                    continue
                try:
                    sm.append(float(p[1]))
                    mx.append(float(p[2]))
                except ValueError:
                    continue
                for nm, v in zip(names[1:], p[5:9]):
                    if v.lower() in ("active", "0x1") or v.lower().startswith("active"):
                        reasons.add(nm)
        try:
            os.remove(self.path)
        except OSError:
            pass
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# across ranks: one independent forest per GPU, no data exchange; the step
# time of the job is the slowest rank's
# ---------------------------------------------------------------------------

PHASES = ("step", "insert", "erase", "knn")


def max_over_ranks(ms, dist, device):
    """Element-wise maximum of the per-phase times over all ranks."""
    import torch
    tt = torch.tensor([float(ms[k]) for k in PHASES], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return dict(zip(PHASES, tt.tolist()))


def rank0_choice(value, dist, device):
    """Rank 0's integer `value` on every rank (an autotuned parameter, so that
    all ranks do the same work)."""
    import torch
    t = torch.tensor([int(value)], dtype=torch.int64, device=device)
    dist.broadcast(t, 0)
    return int(t.item())


def slowest(value, dist, device):
    """The maximum of a per-rank time over all ranks."""
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(ops_per_step_per_rank, world, ms_step):
    """Whole-job rate: every rank's operations over the slowest rank's step time."""
    return ops_per_step_per_rank * world / (ms_step * 1e-3)


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

def run_ours(a, rank, world, dist):
    import torch
    from paper_2112_06188_gb300 import capi
    from paper_2112_06188_gb300.forest import Forest

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    capi.load()
    stream = torch.cuda.Stream(dev)
    # warm-up, timed (profiled), timed again without profiling, end to end
    e2e_warm = min(a.warmup, 3) if a.e2e_steps > 0 else 0
    nsteps = a.warmup + 2 * a.steps + e2e_warm + a.e2e_steps + 1
    W = StepInputs(a.n0, a.batch, a.queries, a.dim, nsteps, seed=2 + 17 * rank)

    def H2D(x):
        return torch.from_numpy(x).to(dev)

    autotune = None
    if a.leaf == "auto":
        from paper_2112_06188_gb300.autotune import CONFIG_CANDIDATES, choose, tune_knn_shape, tune_leaf_size
        t0 = time.perf_counter()
        # the tuning forest and steps come from a seed of their own: the
        # timed steps are never seen before they are timed
        TW = StepInputs(a.n0, a.batch, a.queries, a.dim, 9, seed=7919 + 17 * rank)
        with torch.cuda.stream(stream):
            tsteps = [(H2D(i), H2D(e), H2D(q)) for (i, e, q) in TW.steps]
            best, ms_by_leaf = tune_leaf_size(a.dim, H2D(TW.initial), tsteps, a.k, device=dev, stream=stream,
                                              split=a.split)
        del tsteps
        if dist:
            best = rank0_choice(best, dist, dev)
        a.leaf = best
        t1 = time.perf_counter()
        with torch.cuda.stream(stream):   # then the k-NN launch shape on a forest of that leaf size
            tsteps = [(H2D(i), H2D(e), H2D(q)) for (i, e, q) in TW.steps[:4]]
            shape, ms_by_shape = tune_knn_shape(a.dim, best, H2D(TW.initial), tsteps, a.k, device=dev,
                                                stream=stream, split=a.split)
        del tsteps, TW
        if dist:
            code = rank0_choice(shape[0] * 1000 + shape[1], dist, dev)
            shape = (code // 1000, code % 1000)
        a.knn_shape = "%dx%d" % shape
        autotune = {"candidates_ms_per_step": {str(L): round(v, 3) for L, v in ms_by_leaf.items()},
                    "chosen": best, "tuning_s": round(t1 - t0, 2),
                    "inputs": "own seed (7919), 8 timed steps after one warm-up; not the timed steps",
                    "config_set": {"candidates": list(CONFIG_CANDIDATES),
                                   "chosen": choose({L: ms_by_leaf[L] for L in CONFIG_CANDIDATES})},
                    "knn_shape": shape_record(shape, ms_by_shape, time.perf_counter() - t1,
                                              "the tuning seed's first 4 steps applied, then their "
                                              "4 query batches per shape, 2 rounds after one warm-up round")}
    a.leaf = int(a.leaf)
    shape = parse_shape(a.knn_shape)
    with torch.cuda.stream(stream):
        f = Forest(a.dim, leaf_size=a.leaf, buffer_size=1024, stream=stream, device=dev, split=a.split)
        f.set_knn_shape(*shape)
        f.insert(H2D(W.initial))
        dev_steps = [(H2D(i), H2D(e), H2D(q)) for (i, e, q) in W.steps]
        out_ids = torch.empty((a.queries, a.k), dtype=torch.int32, device=dev)
        out_d2 = torch.empty((a.queries, a.k), dtype=torch.int64, device=dev)
        flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
        counts = torch.zeros(3, dtype=torch.int64, device=dev)
    stream.synchronize()

    def step(i):
        ins, era, q = dev_steps[i]
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        ev[0].record(stream)
        f.insert(ins)
        ev[1].record(stream)
        f.erase(era)
        ev[2].record(stream)
        f.knn(q, a.k, out=(out_ids, out_d2))
        ev[3].record(stream)
        return ev

    def phase_ms(evs):
        t_ins = [e[0].elapsed_time(e[1]) for e in evs]
        t_era = [e[1].elapsed_time(e[2]) for e in evs]
        t_knn = [e[2].elapsed_time(e[3]) for e in evs]
        t_step = [x + y + z for x, y, z in zip(t_ins, t_era, t_knn)]
        return {"step": statistics.mean(t_step), "insert": statistics.mean(t_ins),
                "erase": statistics.mean(t_era), "knn": statistics.mean(t_knn)}, t_step

    for i in range(a.warmup):
        with torch.cuda.stream(stream):
            flush.zero_()
        step(i)
    stream.synchronize()

    clocks = ClockSampler(dev.index)
    if dist:
        dist.barrier()
    torch.cuda.synchronize(dev)
    clocks.start()
    capi.bdl_profile(True)
    evs = []
    t0 = time.perf_counter()
    for i in range(a.warmup, a.warmup + a.steps):
        with torch.cuda.stream(stream):
            flush.zero_()
        evs.append(step(i))
        # this step's k-NN visits, by the counting instance on the same forest
        # and queries, after the step's last event (outside the timed intervals)
        f.knn_count(dev_steps[i][2], a.k, counts, out=(out_ids, out_d2))
    torch.cuda.synchronize(dev)
    wall = time.perf_counter() - t0
    prof = capi.bdl_profile_read_bytes()
    capi.bdl_profile(False)
    clk = clocks.stop()
    if dist:
        dist.barrier()
    # the step's own launches (the counting runs are not part of it)
    launches = sum(v[1] for kname, v in prof.items() if kname != "k_knn_count")
    prof = {kname: v for kname, v in prof.items() if kname != "k_knn_count"}
    ms, t_steps = phase_ms(evs)
    if dist:
        ms = max_over_ranks(ms, dist, dev)
    nodes, points, nq = (int(x) for x in counts.cpu().tolist())

    # the same steps without per-launch profiling events, on the next inputs
    evs2 = []
    for i in range(a.warmup + a.steps, a.warmup + 2 * a.steps):
        with torch.cuda.stream(stream):
            flush.zero_()
        evs2.append(step(i))
    torch.cuda.synchronize(dev)
    ms_plain, _ = phase_ms(evs2)
    if dist:
        ms_plain = max_over_ranks(ms_plain, dist, dev)

    # end to end through the public API from pinned host buffers: every step's
    # inputs are copied in and its k-NN rows copied out inside the timed
    # region.  Steps are pipelined the way a server would run them: the next
    # step's inputs come in and the previous step's rows go out on copy
    # streams while a step computes (two device buffer sets, events between).
    e2e_ms = []
    h2d = d2h = 0
    K = a.e2e_steps
    if K > 0:
        import torch as _t
        first = a.warmup + 2 * a.steps
        # e2e_warm untimed steps through the same loop and buffers first (each
        # with its own inputs): the loop's one-time costs stay out of the timing
        idx = list(range(first, first + e2e_warm + K))
        hin = [tuple(_t.from_numpy(x).pin_memory() for x in W.steps[i]) for i in idx]
        hout = [(_t.empty((a.queries, a.k), dtype=_t.int32).pin_memory(),
                 _t.empty((a.queries, a.k), dtype=_t.int64).pin_memory()) for _ in range(2)]
        din = [tuple(_t.empty_like(x, device=dev) for x in hin[0]) for _ in range(2)]
        dout = [(_t.empty((a.queries, a.k), dtype=_t.int32, device=dev),
                 _t.empty((a.queries, a.k), dtype=_t.int64, device=dev)) for _ in range(2)]
        h2s, d2s = _t.cuda.Stream(dev), _t.cuda.Stream(dev)
        ev_in = [_t.cuda.Event() for _ in range(2)]     # inputs of buffer set b arrived
        ev_used = [_t.cuda.Event() for _ in range(2)]   # the step on set b has finished its k-NN
        ev_out = [_t.cuda.Event() for _ in range(2)]    # rows of set b copied out

        def load(j):
            b = j & 1
            h2s.wait_event(ev_used[b])                  # set b's previous step is done with it
            with _t.cuda.stream(h2s):
                for xd, xh in zip(din[b], hin[j]):
                    xd.copy_(xh, non_blocking=True)
            ev_in[b].record(h2s)

        def e2e_pass(j0, n):
            _t.cuda.synchronize(dev)
            t0 = time.perf_counter()
            load(j0)
            for j in range(j0, j0 + n):
                b = j & 1
                if j + 1 < j0 + n:
                    load(j + 1)
                stream.wait_event(ev_in[b])
                with _t.cuda.stream(stream):
                    flush.zero_()
                f.insert(din[b][0])
                f.erase(din[b][1])
                stream.wait_event(ev_out[b])            # set b's previous rows are out
                f.knn(din[b][2], a.k, out=dout[b])
                ev_used[b].record(stream)
                d2s.wait_event(ev_used[b])
                with _t.cuda.stream(d2s):
                    hout[b][0].copy_(dout[b][0], non_blocking=True)
                    hout[b][1].copy_(dout[b][1], non_blocking=True)
                ev_out[b].record(d2s)
            d2s.synchronize()
            stream.synchronize()
            return (time.perf_counter() - t0) * 1e3 / n

        if e2e_warm:
            e2e_pass(0, e2e_warm)
        e2e_ms.append(e2e_pass(e2e_warm, K))
        if dist:   # the slowest rank's time, as for the device-timed steps
            e2e_ms[-1] = slowest(e2e_ms[-1], dist, dev)
        h2d = sum(x.numel() * x.element_size() for x in hin[0])
        d2h = hout[0][0].numel() * 4 + hout[0][1].numel() * 8   # the k-NN rows (insert ids are known)
    f.close()

    ops_per_step = 2 * a.batch + a.queries
    res = {
        "ms": ms, "ms_plain": ms_plain, "t_steps": t_steps, "launches": launches, "prof": prof,
        "clocks": clk, "wall": wall, "knn_stats": (nodes, points, nq),
        "e2e_ms": statistics.mean(e2e_ms) if e2e_ms else None,
        "h2d": h2d, "d2h": d2h, "ops_per_step": ops_per_step, "autotune": autotune,
    }
    return res


# ---------------------------------------------------------------------------
# batched forests
# ---------------------------------------------------------------------------

def forests_config(a, n_gpus):
    return {"workload": "%d independent forests, dim 2 or 3, sizes log-uniform in [1000, 200000], "
                        "uniform int32 points; per step per forest insert 5-20%% of its size, erase "
                        "2-10%% of its live ids, k=%d NN for 1000-5000 live-set queries" % (a.forests, a.k),
            "forests": a.forests, "k": a.k, "leaf_size": a.leaf, "knn_shape": a.knn_shape, "buffer_size": 1024,
            "l2": "flushed between steps (256 MB write), inputs resident in HBM",
            "parallelism": "one independent set of forests per GPU" if n_gpus > 1 else "single GPU"}


class FlatInputs:
    """One step's per-forest inputs packed into flat device tensors, with the
    pointer and size arrays the batched C entry points take."""

    def __init__(self, step, k, dev):
        import ctypes
        import torch
        self.n_ins = [len(i) for i, _, _ in step]
        self.n_era = [len(e) for _, e, _ in step]
        self.m = [len(q) for _, _, q in step]
        self.ins = torch.from_numpy(np.concatenate([i.ravel() for i, _, _ in step])).to(dev)
        self.era = torch.from_numpy(np.concatenate([e for _, e, _ in step])).to(dev)
        self.q = torch.from_numpy(np.concatenate([q.ravel() for _, _, q in step])).to(dev)
        M = sum(self.m)
        self.oi = torch.empty(M * k, dtype=torch.int32, device=dev)
        self.od = torch.empty(M * k, dtype=torch.int64, device=dev)

        def ptrs(t, counts, width):
            base, es, out, o = t.data_ptr(), t.element_size(), [], 0
            for c, w in zip(counts, width):
                out.append(base + o * es if c else None)
                o += c * w
            return out

        dims = [i.shape[1] for i, _, _ in step]
        self.p_ins = ptrs(self.ins, self.n_ins, dims)
        self.p_era = ptrs(self.era, self.n_era, [1] * len(step))
        self.p_q = ptrs(self.q, self.m, dims)
        self.p_oi = ptrs(self.oi, self.m, [k] * len(step))
        self.p_od = ptrs(self.od, self.m, [k] * len(step))
        A = lambda xs, T=ctypes.c_void_p: (T * len(xs))(*xs)
        self.c_ins, self.c_era, self.c_q = A(self.p_ins), A(self.p_era), A(self.p_q)
        self.c_oi, self.c_od = A(self.p_oi), A(self.p_od)
        self.c_nins, self.c_nera, self.c_m = (A(self.n_ins, ctypes.c_int64), A(self.n_era, ctypes.c_int64),
                                              A(self.m, ctypes.c_int64))
        self.c_null = A([None] * len(step))
        self.c_erased = (ctypes.c_int64 * len(step))()
        self.ops = sum(self.n_ins) + sum(self.n_era) + M


def run_forests(a, rank, world, dist):
    import ctypes
    import torch
    from paper_2112_06188_gb300 import capi, inputs
    from paper_2112_06188_gb300.forest import Forest

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    L = capi.load()
    stream = torch.cuda.Stream(dev)
    sh = ctypes.c_void_p(stream.cuda_stream)
    W = inputs.ForestsWorkload(nf=a.forests, seed=4 + 17 * rank)
    # warm-up, timed (no per-launch events), then P more batched steps with
    # every launch bracketed by events (the per-kernel times; not timed)
    P = min(a.steps, 5)
    nsteps = a.warmup + a.steps + P
    tend = a.warmup + a.steps
    steps = [W.step() for _ in range(nsteps)]
    nf = a.forests
    autotune = None
    if a.leaf == "auto" and nsteps < 2:
        a.leaf = 16                      # too few steps to time a candidate: the default
    if a.leaf == "auto":
        from paper_2112_06188_gb300.autotune import tune_knn_shape_forests, tune_leaf_size_forests
        t0 = time.perf_counter()
        T = lambda x: torch.from_numpy(np.ascontiguousarray(x)).to(dev)
        # forests and steps of a seed of their own: the timed steps are never
        # seen before they are timed
        TW = inputs.ForestsWorkload(nf=a.forests, seed=7919 + 17 * rank)
        tw_steps = [TW.step() for _ in range(4)]
        with torch.cuda.stream(stream):
            tinit = [T(p) for p in TW.initial]
            tsteps = [[(T(i), T(e), T(q)) for i, e, q in st] for st in tw_steps]
            best, ms_by_leaf = tune_leaf_size_forests(TW.dims, tinit, tsteps, a.k, device=dev, stream=stream)
        if dist:
            best = rank0_choice(best, dist, dev)
        t1 = time.perf_counter()
        with torch.cuda.stream(stream):
            shape, ms_by_shape = tune_knn_shape_forests(TW.dims, best, tinit, tsteps, a.k, device=dev,
                                                        stream=stream)
        del tinit, tsteps, tw_steps
        if dist:
            code = rank0_choice(shape[0] * 1000 + shape[1], dist, dev)
            shape = (code // 1000, code % 1000)
        a.leaf = best
        a.knn_shape = "%dx%d" % shape
        autotune = {"candidates_ms_per_step": {str(L): round(v, 3) for L, v in ms_by_leaf.items()},
                    "chosen": best, "tuning_s": round(t1 - t0, 2),
                    "inputs": "forests and steps of their own seed (7919); not the timed steps",
                    "knn_shape": shape_record(shape, ms_by_shape, time.perf_counter() - t1,
                                              "the tuning forests after 4 batched steps, then the 4 steps' "
                                              "query sets per shape, 2 rounds after one warm-up round")}
    a.leaf = int(a.leaf)
    shape = parse_shape(a.knn_shape)
    with torch.cuda.stream(stream):
        A = [Forest(d, leaf_size=a.leaf, stream=stream, device=dev) for d in W.dims]
        B = [Forest(d, leaf_size=a.leaf, stream=stream, device=dev) for d in W.dims]
        for f in A + B:
            f.set_knn_shape(*shape)
        hA = (ctypes.c_void_p * nf)(*[f._h for f in A])
        hB = [f._h for f in B]
        init = FlatInputs([(p, np.zeros(0, np.int32), np.zeros((0, p.shape[1]), np.int32))
                           for p in W.initial], a.k, dev)
        flat = [FlatInputs(st, a.k, dev) for st in steps]
        flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream.synchronize()
    capi.check(L.bdl_insert_batch(hA, nf, init.c_ins, init.c_nins, init.c_null, sh), "bdl_insert_batch")
    for i in range(nf):
        capi.check(L.bdl_insert(hB[i], init.p_ins[i], init.n_ins[i], None, sh), "bdl_insert")
    stream.synchronize()
    del init

    def batched(x):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        ev[0].record(stream)
        capi.check(L.bdl_insert_batch(hA, nf, x.c_ins, x.c_nins, x.c_null, sh), "bdl_insert_batch")
        ev[1].record(stream)
        capi.check(L.bdl_erase_batch(hA, nf, x.c_era, x.c_nera, x.c_erased, sh), "bdl_erase_batch")
        ev[2].record(stream)
        capi.check(L.bdl_knn_batch(hA, nf, x.c_q, x.c_m, a.k, x.c_oi, x.c_od, sh), "bdl_knn_batch")
        ev[3].record(stream)
        return ev

    def per_forest(x, oi, od):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        n = ctypes.c_int64(0)
        ev[0].record(stream)
        for i in range(nf):
            capi.check(L.bdl_insert(hB[i], x.p_ins[i], x.n_ins[i], None, sh), "bdl_insert")
        ev[1].record(stream)
        for i in range(nf):
            capi.check(L.bdl_erase(hB[i], x.p_era[i], x.n_era[i], ctypes.byref(n), sh), "bdl_erase")
        ev[2].record(stream)
        for i in range(nf):
            capi.check(L.bdl_knn(hB[i], x.p_q[i], x.m[i], a.k, oi[i], od[i], sh), "bdl_knn")
        ev[3].record(stream)
        return ev

    # per-forest outputs go to their own buffers so that the arms can be compared
    outB = []
    for x in flat:
        oi = torch.empty_like(x.oi)
        od = torch.empty_like(x.od)
        off, pi, pd = 0, [], []
        for m in x.m:
            pi.append(oi.data_ptr() + off * a.k * 4 if m else None)
            pd.append(od.data_ptr() + off * a.k * 8 if m else None)
            off += m
        outB.append((oi, od, pi, pd))

    def flush_l2():
        with torch.cuda.stream(stream):
            flush.zero_()

    for i in range(a.warmup):
        flush_l2()
        batched(flat[i])
        flush_l2()
        per_forest(flat[i], outB[i][2], outB[i][3])
    stream.synchronize()

    clocks = ClockSampler(dev.index)
    if dist:
        dist.barrier()
    torch.cuda.synchronize(dev)
    clocks.start()
    l0 = capi.bdl_launch_count()
    evA = []
    for i in range(a.warmup, tend):
        flush_l2()
        evA.append(batched(flat[i]))
    torch.cuda.synchronize(dev)
    launchesA = capi.bdl_launch_count() - l0
    clk = clocks.stop()
    if dist:
        dist.barrier()
    l0 = capi.bdl_launch_count()
    evB = []
    for i in range(a.warmup, tend):
        flush_l2()
        evB.append(per_forest(flat[i], outB[i][2], outB[i][3]))
    torch.cuda.synchronize(dev)
    launchesB = capi.bdl_launch_count() - l0
    same_forests = all(f.size() == g.size() and f.tree_mask() == g.tree_mask() for f, g in zip(A, B))
    # the profiled steps (batched arm only, after the timed ones)
    capi.bdl_profile(True)
    evP = []
    for i in range(tend, nsteps):
        flush_l2()
        evP.append(batched(flat[i]))
    torch.cuda.synchronize(dev)
    prof = capi.bdl_profile_read()
    capi.bdl_profile(False)

    def phases(evs):
        t = [[e[j].elapsed_time(e[j + 1]) for e in evs] for j in range(3)]
        ms = {"insert": sum(t[0]) / len(evs), "erase": sum(t[1]) / len(evs), "knn": sum(t[2]) / len(evs)}
        ms["step"] = ms["insert"] + ms["erase"] + ms["knn"]
        return ms

    msA, msB, msP = phases(evA), phases(evB), phases(evP)
    if dist:
        msA, msB = max_over_ranks(msA, dist, dev), max_over_ranks(msB, dist, dev)
    identical = same_forests and all(torch.equal(flat[i].oi, outB[i][0]) and torch.equal(flat[i].od, outB[i][1])
                                     for i in range(a.warmup, tend))
    # read-only repeats of the last step's k-NN on the final forests: the
    # batched call, a prepared plan (kernels only), and that plan replayed
    # from a CUDA graph; all must give the same rows
    x = flat[-1]
    R = 20
    ref_i, ref_d = x.oi.clone(), x.od.clone()

    def rep_ms(fn):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        stream.synchronize()
        e0.record(stream)
        for _ in range(R):
            fn()
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1) / R

    eager_ms = rep_ms(lambda: capi.check(L.bdl_knn_batch(hA, nf, x.c_q, x.c_m, a.k, x.c_oi, x.c_od, sh),
                                         "bdl_knn_batch"))
    same_eager = torch.equal(x.oi, ref_i) and torch.equal(x.od, ref_d)
    st, plan = capi.bdl_knn_plan_create(list(hA), x.p_q, x.m, a.k, x.p_oi, x.p_od, sh)
    capi.check(st, "bdl_knn_plan_create")
    plan_ms = rep_ms(lambda: capi.check(L.bdl_knn_plan_launch(plan, sh), "bdl_knn_plan_launch"))
    same_plan = torch.equal(x.oi, ref_i) and torch.equal(x.od, ref_d)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        capi.check(L.bdl_knn_plan_launch(plan, ctypes.c_void_p(stream.cuda_stream)), "bdl_knn_plan_launch")
    x.oi.fill_(-1)
    def replay():
        with torch.cuda.stream(stream):    # replays run on the current stream
            g.replay()

    graph_ms = rep_ms(replay)
    same_graph = torch.equal(x.oi, ref_i) and torch.equal(x.od, ref_d)
    del g
    capi.bdl_knn_plan_destroy(plan)
    knn_repeat = {"queries": sum(x.m), "batched_call_ms": round(eager_ms, 3), "prepared_plan_ms": round(plan_ms, 3),
                  "cuda_graph_replay_ms": round(graph_ms, 3),
                  "identical_results": bool(same_eager and same_plan and same_graph)}
    x = flat[tend - 1]
    res = {"msA": msA, "msB": msB, "msP": msP, "P": P, "launchesA": launchesA // a.steps,
           "launchesB": launchesB // a.steps,
           "prof": prof, "clocks": clk, "identical": bool(identical), "knn_repeat": knn_repeat,
           "ops": sum(flat[i].ops for i in range(a.warmup, tend)) / a.steps,
           "inserted": sum(x.n_ins), "erased": sum(x.n_era), "queries": sum(x.m), "autotune": autotune,
           "points": int(sum(f.size() for f in A))}
    for f in A + B:
        f.close()
    return res


def forests_cpu_sample(a, nsample=16):
    """The oracle on the first `nsample` forests of the same workload, one step."""
    from oracle.oracle import OracleForest
    from paper_2112_06188_gb300 import inputs
    W = inputs.ForestsWorkload(nf=a.forests, seed=4)
    step = W.step()
    nsample = min(nsample, a.forests)
    os_ = []
    for i in range(nsample):
        o = OracleForest(W.dims[i], leaf_size=16, buffer_size=1024)
        o.insert(W.initial[i])
        os_.append(o)
    t0 = time.perf_counter()
    ops = 0
    for i in range(nsample):
        ins, era, q = step[i]
        os_[i].insert(ins)
        os_[i].erase(era)
        os_[i].knn(q, a.k)
        ops += len(ins) + len(era) + len(q)
    dt = time.perf_counter() - t0
    sample = "one step on the first %d of the %d forests, one host core" % (nsample, a.forests)
    return ops / dt, sample


def report_forests(a, res, world):
    msA, msB = res["msA"], res["msB"]
    value = res["ops"] * world / (msA["step"] * 1e-3)
    out = {
        "metric": METRIC, "value": round(value, 1), "unit": "ops/s", "n_gpus": world,
        "steps": a.steps, "warmup": a.warmup, "ms_per_step": round(msA["step"], 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
        "data": "synthetic", "config": dict(forests_config(a, world), leaf_autotune=res["autotune"]),
        "phase_ms": {k: round(v, 3) for k, v in msA.items()},
        "per_forest_calls": {"value": round(res["ops"] * world / (msB["step"] * 1e-3), 1), "unit": "ops/s",
                             "phase_ms": {k: round(v, 3) for k, v in msB.items()},
                             "gpu_launches": res["launchesB"]},
        "speedup_vs_per_forest": round(msB["step"] / msA["step"], 2),
        "identical_results": res["identical"],
        "knn_repeat_final_forests": res["knn_repeat"],
        "per_step": {"inserted": res["inserted"], "erased": res["erased"], "queries": res["queries"],
                     "live_points_after": res["points"]},
        "gpu_launches": res["launchesA"],
        "kernel_ms": {k: [round(v[0] / res["P"], 4), v[1] // res["P"]] for k, v in
                      sorted(res["prof"].items(), key=lambda kv: -kv[1][0])},
        "profiling": "the timed steps run without per-launch events; kernel_ms comes from %d more batched "
                     "steps after them with every launch bracketed by CUDA events (profiled_phase_ms: "
                     "those steps' own phase times)" % res["P"],
        "profiled_phase_ms": {k: round(v, 3) for k, v in res["msP"].items()},
        "clocks": res["clocks"],
    }
    if world == 1 and not a.no_cpu_baseline:
        v, sample = forests_cpu_sample(a)
        out["cpu_baseline"] = {"value": round(v, 1), "unit": "ops/s", "cores": 1, "kind": "oracle",
                               "sample": sample}
    return out


# ---------------------------------------------------------------------------
# serving
# ---------------------------------------------------------------------------

SERVE_HBM_BUDGET = 24 << 30       # the forest's own device memory
SERVE_STAGING = 2 << 30           # requests' buffers in flight


def serve_config(a):
    return {"workload": "serving: one 5-D forest growing from 1M to %d uniform int32 points under "
                        "Poisson arrivals (%.0f requests/s) of inserts (1k-1M points), erases (1k-500k "
                        "live ids) and k-NN (1-100k queries, k in {1,5,10}) in a 4:1:5 mix, sizes "
                        "log-uniform" % (a.n_final, a.rate),
            "dim": 5, "n0": 1_000_000, "n_final": a.n_final, "rate_per_s": a.rate,
            "hbm_budget_bytes": SERVE_HBM_BUDGET, "staging_budget_bytes": SERVE_STAGING,
            "leaf_size": 16, "buffer_size": 1024, "l2": "not flushed (requests stream continuously)",
            "parallelism": "single GPU"}


def serve_once(a, reqs, initial, serial, paced, dev):
    """Run the request list through a server; returns per-request results,
    the makespan (s) and the number of device groups."""
    import threading
    import torch
    from paper_2112_06188_gb300.forest import Forest
    from paper_2112_06188_gb300.serve import Server
    f = Forest(5, leaf_size=16, buffer_size=1024, hbm_budget_bytes=SERVE_HBM_BUDGET, device=dev)
    f.insert(torch.from_numpy(initial).to(dev))
    torch.cuda.synchronize(dev)
    # outputs allocated (pinned) up front, so that submitting costs nothing
    outs = []
    for _, kind, payload, k in reqs:
        if kind == "insert":
            outs.append(torch.empty(payload.shape[0], dtype=torch.int32).pin_memory())
        elif kind == "knn":
            outs.append((torch.empty((payload.shape[0], k), dtype=torch.int32).pin_memory(),
                         torch.empty((payload.shape[0], k), dtype=torch.int64).pin_memory()))
        else:
            outs.append(None)
    srv = Server(f, serial=serial, staging_budget_bytes=SERVE_STAGING, max_inflight=256)
    tickets = [None] * len(reqs)
    lateness = []
    start = [0.0]

    def submitter():
        # request i arrives at start + t_i on the server's clock; latency is
        # counted from that arrival, so a late submit cannot hide queueing
        t0 = start[0] = srv.now_ms()
        for i, (t, kind, payload, k) in enumerate(reqs):
            if paced:
                dt = t * 1e3 - (srv.now_ms() - t0)
                if dt > 0:
                    time.sleep(dt * 1e-3)
                lateness.append(srv.now_ms() - t0 - t * 1e3)
            if kind == "insert":
                tickets[i] = srv.insert(payload, out=outs[i])
            elif kind == "erase":
                tickets[i] = srv.erase(payload)
            else:
                tickets[i] = srv.knn(payload, k, out=outs[i])

    t0 = time.perf_counter()
    th = threading.Thread(target=submitter)
    th.start()
    th.join()
    res = [srv.wait(t) for t in tickets]
    makespan = time.perf_counter() - t0
    for (t, _, _, _), r in zip(reqs, res):
        r["t_arrival_ms"] = start[0] + (t * 1e3 if paced else 0.0)
    groups = srv.groups()
    srv.close()
    live = f.size()
    f.close()
    return res, makespan, groups, live, lateness


def latency_summary(reqs, res):
    out = {}
    for kind in ("insert", "erase", "knn"):
        lat = [r["t_done_ms"] - r["t_arrival_ms"] for (_, kd, _, _), r in zip(reqs, res) if kd == kind]
        if lat:
            out[kind] = {"p50_ms": round(float(np.percentile(lat, 50)), 3),
                         "p99_ms": round(float(np.percentile(lat, 99)), 3), "count": len(lat)}
    return out


def run_serve(a):
    import torch
    from paper_2112_06188_gb300 import capi, inputs
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    capi.load()
    W = inputs.ServeWorkload(dim=5, n0=1_000_000, n_final=a.n_final, rate=a.rate, seed=5)
    reqs = [(t, kind, torch.from_numpy(np.ascontiguousarray(p)).pin_memory(), k)
            for t, kind, p, k in W.requests()]
    initial = W.initial
    n_ins = sum(p.shape[0] for _, kd, p, _ in reqs if kd == "insert")
    n_era = sum(p.shape[0] for _, kd, p, _ in reqs if kd == "erase")
    n_q = sum(p.shape[0] for _, kd, p, _ in reqs if kd == "knn")
    # warm-up: a short prefix, not timed
    serve_once(a, reqs[:20], initial, serial=False, paced=False, dev=dev)
    clocks = ClockSampler(dev.index)
    clocks.start()
    l0 = capi.bdl_launch_count()
    res, span, groups, live, late = serve_once(a, reqs, initial, serial=False, paced=True, dev=dev)
    launches = capi.bdl_launch_count() - l0
    clk = clocks.stop()
    res_s, span_s, groups_s, live_s, _ = serve_once(a, reqs, initial, serial=True, paced=True, dev=dev)
    # saturated: every request queued at once (sustained throughput)
    res_b, span_b, groups_b, _, _ = serve_once(a, reqs, initial, serial=False, paced=False, dev=dev)
    res_bs, span_bs, _, _, _ = serve_once(a, reqs, initial, serial=True, paced=False, dev=dev)

    def same(r1, r2):
        for (_, kind, _, _), x, y in zip(reqs, r1, r2):
            if x["status"] != y["status"] or x["n_done"] != y["n_done"]:
                return False
            if kind == "knn" and not (torch.equal(x["ids"], y["ids"]) and torch.equal(x["d2"], y["d2"])):
                return False
            if kind == "insert" and not torch.equal(x["ids"], y["ids"]):
                return False
        return True

    identical = same(res, res_s) and same(res, res_b) and same(res, res_bs)
    ok = all(r["status"] == 0 for r in res)
    ops = n_ins + n_era + n_q
    value = ops / span_b
    out = {
        "metric": METRIC, "value": round(value, 1), "unit": "ops/s", "n_gpus": 1,
        "steps": 1, "warmup": 1, "ms_per_step": round(span_b * 1e3, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": serve_config(a),
        "requests": {"total": len(reqs), "insert": sum(1 for r in reqs if r[1] == "insert"),
                     "erase": sum(1 for r in reqs if r[1] == "erase"),
                     "knn": sum(1 for r in reqs if r[1] == "knn"),
                     "points_inserted": n_ins, "ids_erased": n_era, "queries": n_q,
                     "live_points_after": live},
        "sustained": {"updates_per_s": round((n_ins + n_era) / span_b, 1), "queries_per_s": round(n_q / span_b, 1),
                      "makespan_s": round(span_b, 4), "device_groups": groups_b,
                      "one_at_a_time": {"updates_per_s": round((n_ins + n_era) / span_bs, 1),
                                        "queries_per_s": round(n_q / span_bs, 1),
                                        "makespan_s": round(span_bs, 4)}},
        "latency": {"continuous_batching": latency_summary(reqs, res),
                    "one_at_a_time": latency_summary(reqs, res_s),
                    "offered_span_s": round(reqs[-1][0], 4), "served_span_s": round(span, 4),
                    "served_span_one_at_a_time_s": round(span_s, 4),
                    "device_groups": groups, "device_groups_one_at_a_time": groups_s,
                    "latency_from": "arrival time (Poisson schedule on the server's clock)",
                    "submit_lateness_p99_ms": round(float(np.percentile(late, 99)), 3) if late else None},
        "identical_results": bool(identical), "all_ok": bool(ok),
        "gpu_launches": launches,
        "clocks": clk,
    }
    if not a.no_cpu_baseline:
        out["cpu_baseline"] = serve_cpu_sample(a)
    return out


def serve_cpu_sample(a, n_req=40):
    """The oracle replaying the first requests of the same stream on a forest
    of 1/10 the initial size (requests at 1/10 scale), one host core."""
    from oracle.oracle import OracleForest
    from paper_2112_06188_gb300 import inputs
    W = inputs.ServeWorkload(dim=5, n0=100_000, n_final=10 ** 9, rate=a.rate, seed=5,
                             ins=(100, 100_000), dele=(100, 50_000), knn=(1, 10_000), max_requests=n_req)
    o = OracleForest(5, leaf_size=16, buffer_size=1024)
    o.insert(W.initial)
    ops, t = 0, 0.0
    for _, kind, p, k in W.requests():
        t0 = time.perf_counter()
        if kind == "insert":
            o.insert(p)
        elif kind == "erase":
            o.erase(p)
        else:
            o.knn(p, k)
        t += time.perf_counter() - t0
        ops += len(p)
    return {"value": round(ops / t, 1), "unit": "ops/s", "cores": 1, "kind": "oracle",
            "sample": "first %d requests of the same stream at 1/10 scale (forest of 100k points), "
                      "one host core" % n_req}


# ---------------------------------------------------------------------------
# sweeps: batch size (inserts, erases) and k
# ---------------------------------------------------------------------------

SWEEP_BATCHES = (10_000, 100_000, 1_000_000, 2_000_000, 3_000_000, 4_000_000, 5_000_000)
SWEEP_KS = tuple(range(2, 12))


def run_sweep(a):
    import torch
    from paper_2112_06188_gb300 import capi, inputs
    from paper_2112_06188_gb300.forest import Forest
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    capi.load()
    stream = torch.cuda.Stream(dev)
    n = 10_000_000
    sets = {"2-D clusters": (2, inputs.gaussian_clusters(n, 2, seed=21)),
            "7-D uniform": (7, inputs.uniform_points(n, 7, seed=22)),
            "7-D clusters": (7, inputs.gaussian_clusters(n, 7, seed=23))}

    def timed(fn):
        a_ = torch.cuda.Event(enable_timing=True)
        b_ = torch.cuda.Event(enable_timing=True)
        stream.synchronize()
        a_.record(stream)
        fn()
        b_.record(stream)
        b_.synchronize()
        return a_.elapsed_time(b_)

    out = {"insert_updates_per_s": {}, "erase_updates_per_s": {}, "knn_queries_per_s": {}}
    clocks = ClockSampler(dev.index)
    clocks.start()
    for name, (dim, pts) in sets.items():
        P = torch.from_numpy(pts).to(dev)
        ins, era, kq = {}, {}, {}
        for b in SWEEP_BATCHES:
            with torch.cuda.stream(stream):
                f = Forest(dim, stream=stream, device=dev, split=a.split)
                ms = timed(lambda: [f.insert(P[i:i + b]) for i in range(0, n, b)])
                ins[b] = round(n / (ms * 1e-3), 1)
                ids = torch.from_numpy(np.random.default_rng(b).permutation(n).astype(np.int32)).to(dev)
                ms = timed(lambda: [f.erase(ids[i:i + b]) for i in range(0, n, b)])
                era[b] = round(n / (ms * 1e-3), 1)
                assert f.size() == 0
                f.close()
        with torch.cuda.stream(stream):
            f = Forest(dim, stream=stream, device=dev, split=a.split)
            step = n // 20
            for i in range(0, n, step):
                f.insert(P[i:i + step])
            oi = torch.empty((n, max(SWEEP_KS)), dtype=torch.int32, device=dev)
            od = torch.empty((n, max(SWEEP_KS)), dtype=torch.int64, device=dev)
            f.knn(P[:100_000], 2)          # warm-up (buffer tree)
            for k in SWEEP_KS:
                ok, dk = oi[:, :k].contiguous(), od[:, :k].contiguous()
                ms = timed(lambda: f.knn(P, k, out=(ok, dk)))
                kq[k] = round(n / (ms * 1e-3), 1)
            f.close()
        out["insert_updates_per_s"][name] = ins
        out["erase_updates_per_s"][name] = era
        out["knn_queries_per_s"][name] = kq
        del P
    clk = clocks.stop()
    best = max(v for d in out["knn_queries_per_s"].values() for v in d.values())
    return {"metric": METRIC, "value": best, "unit": "queries/s", "n_gpus": 1, "steps": 1, "warmup": 0,
            "ms_per_step": None, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "int64", "data": "synthetic",
            "config": {"workload": "sweeps on 10M points (2-D clusters, 7-D uniform, 7-D clusters): insert and erase "
                                   "throughput vs batch size, k-NN graph throughput vs k after 5% insert "
                                   "batches", "split": a.split, "leaf_size": 16, "buffer_size": 1024,
                       "batches": list(SWEEP_BATCHES), "ks": list(SWEEP_KS)},
            "sweep": out, "clocks": clk}


def recorded_traffic(kernel, leaf, knn_shape):
    """DRAM bytes per launch of `kernel` from its committed ncu summary, or None
    when the summary is missing, was captured at another leaf size or k-NN
    launch shape, or the kernel source changed since the capture."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "%s_3d_10M.md" % kernel)
    try:
        text = open(path).read()
    except OSError:
        return None
    fields = dict(line.split(": ", 1) for line in text.splitlines()
                  if line.startswith(("kernel_source:", "source_sha256_16:", "dram_bytes_per_launch:",
                                      "leaf_size:", "knn_shape:")))
    if fields.get("leaf_size", "").strip() != str(leaf):
        return None
    if fields.get("knn_shape", "128x32").strip() != knn_shape:
        return None
    try:
        src = open(os.path.join(ROOT, fields["kernel_source"].strip()), "rb").read()
    except (KeyError, OSError):
        return None
    if hashlib.sha256(src).hexdigest()[:16] != fields.get("source_sha256_16", "").strip():
        return None
    return int(fields["dram_bytes_per_launch"])


ROOFLINE_KERNELS = ("k_knn", "k_subtree", "k_build_levels", "k_erase_locate", "k_bloom_build")


def rec_bytes(dim):
    """Bytes of one point record in a tree: d coordinates and the id, padded to
    a multiple of 16 bytes (the leaf scan reads whole records)."""
    return 4 * ((dim + 1 + 3) // 4 * 4)


def rooflines(a, res, peaks):
    """Each hot kernel of the timed region against the measured HBM peak:
    achieved = algorithmic bytes summed over the timed steps / the kernel's
    device time summed over the same steps (CUDA events around every launch).
    The bytes of k_knn come from the counting instance run on every timed
    step's forest and queries (4d + 12k per query, 32 per visited node, one
    record per examined leaf point); the others' from the library's own
    per-launch figures (bdl_profile_read_bytes)."""
    prof = res["prof"]
    peak = peaks.get("hbm_gbs")
    src = "measured (MEASURED_PEAKS.json hbm_gbs)" if "when" in peaks else "fallback"
    nodes, points, nq = res["knn_stats"]
    out = []
    for name in ROOFLINE_KERNELS:
        if name not in prof:
            continue
        tot_ms, nl, algo = prof[name]
        extra = {}
        if name == "k_knn":
            if not nq:
                continue
            algo = nq * (4 * a.dim + 12 * a.k) + 32 * nodes + rec_bytes(a.dim) * points
            extra = {"knn_visits_per_query": {"nodes": round(nodes / nq, 2), "leaf_points": round(points / nq, 2)},
                     "queries_counted": nq}
        if not algo or not tot_ms or not peak:
            continue
        achieved = algo / (tot_ms * 1e-3) / 1e9
        traffic = recorded_traffic(name, a.leaf, a.knn_shape) if a.n0 == 10_000_000 and a.queries == 1_000_000 else None
        e = {"kernel": name, "bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
             "frac": round(achieved / peak, 4), "traffic": traffic, "peak_source": src,
             "ms_per_launch": round(tot_ms / nl, 4), "launches_per_step": round(nl / a.steps, 2),
             "ms_per_step": round(tot_ms / a.steps, 4),
             "algorithmic_bytes_per_launch": int(algo / nl)}
        e.update(extra)
        out.append(e)
    return out


# ---------------------------------------------------------------------------
# CPU oracle (reference arm and cpu_baseline)
# ---------------------------------------------------------------------------

def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo), or None."""
    try:
        txt = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in txt.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return None


def oracle_sample(a, nsteps, seed=2):
    """Time the oracle on a 1/10-scale step: forest of n0/10 points, then per
    step insert batch/10, erase batch/10, k-NN for queries/10.  Returns the
    per-step times, the operations per step, a description, and the last
    step's k-NN rerun on all host cores (queries/s, threads)."""
    from oracle.oracle import OracleForest
    from oracle.threads import oracle_knn
    n0, b, m = a.n0 // 10, a.batch // 10, a.queries // 10
    W = StepInputs(n0, b, m, a.dim, nsteps, seed=seed)
    o = OracleForest(a.dim, leaf_size=16 if a.leaf == "auto" else int(a.leaf), buffer_size=1024, split=a.split)
    o.insert(W.initial)
    times = []
    for ins, era, q in W.steps:
        t0 = time.perf_counter()
        o.insert(ins)
        o.erase(era)
        o.knn(q, a.k)
        times.append(time.perf_counter() - t0)
    ops = 2 * b + m
    sample = ("1/10-scale step on one host core: forest of %d points, insert %d, erase %d, "
              "k=%d NN for %d queries" % (n0, b, b, a.k, m))
    threads = os.cpu_count() or 1
    t0 = time.perf_counter()
    oracle_knn(o, W.steps[-1][2], a.k, threads=threads)
    allc = {"queries_per_s": round(m / (time.perf_counter() - t0), 1), "threads": threads,
            "what": "the last sample step's k-NN batch split over host threads (the oracle's k-NN only reads "
                    "the forest)"}
    return times, ops, sample, allc


def cpu_baseline_line(a):
    """The oracle's cpu_baseline: median of three 1/10-scale steps after one
    warm-up step (the paper's protocol, Sec. VI), on one core."""
    times, ops, sample, allc = oracle_sample(a, 4)
    med = statistics.median(times[1:])
    return {"value": round(ops / med, 1), "unit": "ops/s", "cores": 1, "kind": "oracle",
            "sample": sample + "; median of 3 steps after one warm-up step",
            "step_s": [round(t, 3) for t in times[1:]], "nproc": os.cpu_count(), "cpu_model": cpu_model(),
            "knn_all_cores": allc}


def run_reference(a, rank):
    if rank != 0:
        return
    if a.workload == "serve":
        cb = serve_cpu_sample(a)
        out = {"impl": "reference", "metric": METRIC, "value": cb["value"], "unit": "ops/s",
               "n_gpus": a.gpus, "steps": 1, "warmup": 0, "ms_per_step": None, "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
               "config": serve_config(a), "cpu_baseline": cb,
               "e2e": {"value": cb["value"], "unit": "ops/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(out), flush=True)
        return
    if a.workload == "forests":
        vals = []
        for _ in range(max(1, a.steps)):
            v, sample = forests_cpu_sample(a)
            vals.append(v)
        value = statistics.median(vals)
        out = {"impl": "reference", "metric": METRIC, "value": round(value, 1), "unit": "ops/s",
               "n_gpus": a.gpus, "steps": a.steps, "warmup": a.warmup, "ms_per_step": None,
               "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
               "data": "synthetic", "config": forests_config(a, a.gpus),
               "cpu_baseline": {"value": round(value, 1), "unit": "ops/s", "cores": 1, "kind": "oracle",
                                "sample": sample},
               "e2e": {"value": round(value, 1), "unit": "ops/s", "h2d_bytes_per_step": 0,
                       "d2h_bytes_per_step": 0}}
        print(json.dumps(out), flush=True)
        return
    W = a.warmup
    times, ops, sample, allc = oracle_sample(a, W + a.steps)
    t = times[W:]
    ms = 1e3 * sum(t) / len(t)
    value = ops / (ms * 1e-3)
    out = {"impl": "reference", "metric": METRIC, "value": round(value, 1), "unit": "ops/s",
           "n_gpus": a.gpus, "steps": a.steps, "warmup": a.warmup, "ms_per_step": round(ms, 3),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
           "data": "synthetic", "config": workload_config(a, a.gpus),
           "cpu_baseline": {"value": round(value, 1), "unit": "ops/s", "cores": 1, "kind": "oracle",
                            "sample": sample, "nproc": os.cpu_count(), "cpu_model": cpu_model(),
                            "knn_all_cores": allc},
           "e2e": {"value": round(value, 1), "unit": "ops/s", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    a = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    dist = None
    if a.impl == "reference":
        run_reference(a, rank)
        return
    if world > 1:
        import torch
        import torch.distributed as tdist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        tdist.init_process_group("nccl")
        dist = tdist
    if a.workload == "sweep":
        if rank == 0:
            print(json.dumps(run_sweep(a)), flush=True)
        if dist:
            dist.destroy_process_group()
        return
    if a.workload == "serve":
        if rank == 0:
            print(json.dumps(run_serve(a)), flush=True)
        if dist:
            dist.destroy_process_group()
        return
    if a.workload == "forests":
        res = run_forests(a, rank, world, dist)
        if rank == 0:
            print(json.dumps(report_forests(a, res, world)), flush=True)
        if dist:
            dist.destroy_process_group()
        return
    res = run_ours(a, rank, world, dist)
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            peaks = json.load(fh)
    except Exception:
        peaks = {"hbm_gbs": 6800.0, "source": "fallback"}
    ms = res["ms"]
    ops = res["ops_per_step"] * world
    value = job_throughput(res["ops_per_step"], world, ms["step"])
    out = {
        "metric": METRIC, "value": round(value, 1), "unit": "ops/s", "n_gpus": world,
        "steps": a.steps, "warmup": a.warmup, "ms_per_step": round(ms["step"], 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
        "data": "synthetic", "config": workload_config(a, world),
        "updates_per_s": round(2 * a.batch * world / ((ms["insert"] + ms["erase"]) * 1e-3), 1),
        "queries_per_s": round(a.queries * world / (ms["knn"] * 1e-3), 1),
        "phase_ms": {k: round(v, 3) for k, v in ms.items()},
        "gpu_launches": res["launches"],
        "kernel_ms": {k: [round(v[0] / a.steps, 4), v[1] // a.steps] for k, v in
                      sorted(res["prof"].items(), key=lambda kv: -kv[1][0])},
        "profiling": "every launch of the timed steps bracketed by CUDA events (per-kernel times, rooflines); "
                     "unprofiled_ms_per_step: the next %d steps without them" % a.steps,
        "unprofiled_ms_per_step": round(res["ms_plain"]["step"], 3),
        "unprofiled_phase_ms": {k: round(v, 3) for k, v in res["ms_plain"].items()},
        "step_ms_min_max": [round(min(res["t_steps"]), 3), round(max(res["t_steps"]), 3)],
        "clocks": res["clocks"],
    }
    rl = rooflines(a, res, peaks)
    if rl:
        dom = max(rl, key=lambda e: e["ms_per_step"])
        out["roofline"] = dom
        out["rooflines"] = rl
    if res["autotune"]:
        out["config"]["leaf_autotune"] = res["autotune"]
    if res["e2e_ms"]:
        out["e2e"] = {"value": round(ops / (res["e2e_ms"] * 1e-3), 1), "unit": "ops/s",
                      "h2d_bytes_per_step": res["h2d"], "d2h_bytes_per_step": res["d2h"],
                      "ms_per_step": round(res["e2e_ms"], 3), "steps": a.e2e_steps,
                      "warmup": min(a.warmup, 3),
                      "pipelined": "next inputs in and previous rows out on copy streams during each step"}
    if world == 1 and not a.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline_line(a)
    print(json.dumps(out), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
