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
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "batch updates/sec and k-NN queries/sec at 10M pts; HBM GB/s; serve p50/p99 ms"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n0", type=int, default=10_000_000)
    ap.add_argument("--batch", type=int, default=1_000_000)
    ap.add_argument("--queries", type=int, default=1_000_000)
    ap.add_argument("--k", type=int, default=10)
    ap.add_argument("--dim", type=int, default=3)
    ap.add_argument("--leaf", type=int, default=16)
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    return ap.parse_args()


def workload_config(a, n_gpus):
    return {"workload": "3-D uniform int32 forest of %d points; per step insert %d, erase %d "
                        "live ids, k=%d NN for %d live-set queries" % (a.n0, a.batch, a.batch, a.k, a.queries),
            "dim": a.dim, "n0": a.n0, "insert_batch": a.batch, "erase_batch": a.batch,
            "queries": a.queries, "k": a.k, "leaf_size": a.leaf, "buffer_size": 1024,
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
        self.path = os.path.join(ROOT, "gpurun_out", "clocks_%d.csv" % os.getpid())

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
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
    nsteps = a.warmup + a.steps + a.e2e_steps + 1
    W = StepInputs(a.n0, a.batch, a.queries, a.dim, nsteps, seed=2 + 17 * rank)

    def H2D(x):
        return torch.from_numpy(x).to(dev)

    with torch.cuda.stream(stream):
        f = Forest(a.dim, leaf_size=a.leaf, buffer_size=1024, stream=stream, device=dev)
        f.insert(H2D(W.initial))
        dev_steps = [(H2D(i), H2D(e), H2D(q)) for (i, e, q) in W.steps]
        out_ids = torch.empty((a.queries, a.k), dtype=torch.int32, device=dev)
        out_d2 = torch.empty((a.queries, a.k), dtype=torch.int64, device=dev)
        flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
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
    launches0 = capi.bdl_launch_count()
    evs = []
    t0 = time.perf_counter()
    for i in range(a.warmup, a.warmup + a.steps):
        with torch.cuda.stream(stream):
            flush.zero_()
        evs.append(step(i))
    torch.cuda.synchronize(dev)
    wall = time.perf_counter() - t0
    launches = capi.bdl_launch_count() - launches0
    prof = capi.bdl_profile_read()
    capi.bdl_profile(False)
    clk = clocks.stop()
    if dist:
        dist.barrier()

    t_ins = [e[0].elapsed_time(e[1]) for e in evs]
    t_era = [e[1].elapsed_time(e[2]) for e in evs]
    t_knn = [e[2].elapsed_time(e[3]) for e in evs]
    t_step = [x + y + z for x, y, z in zip(t_ins, t_era, t_knn)]
    ms_step = sum(t_step) / len(t_step)
    ms = {"step": ms_step, "insert": sum(t_ins) / len(t_ins), "erase": sum(t_era) / len(t_era),
          "knn": sum(t_knn) / len(t_knn)}
    if dist:
        ms = max_over_ranks(ms, dist, dev)

    # k-NN visit counts for the algorithmic bytes (separate, untimed launch)
    f.knn_stats(True)
    f.knn(dev_steps[a.warmup + a.steps - 1][2], a.k, out=(out_ids, out_d2))
    stream.synchronize()
    nodes, points, nq = f.knn_stats()
    f.knn_stats(False)

    # end to end through the public API with host buffers, copies timed
    e2e_ms = []
    h2d = d2h = 0
    for i in range(a.warmup + a.steps, a.warmup + a.steps + a.e2e_steps):
        ins, era, q = W.steps[i]
        import torch as _t
        ins_h = _t.from_numpy(ins).pin_memory()
        era_h = _t.from_numpy(era).pin_memory()
        q_h = _t.from_numpy(q).pin_memory()
        oi_h = _t.empty((a.queries, a.k), dtype=_t.int32).pin_memory()
        od_h = _t.empty((a.queries, a.k), dtype=_t.int64).pin_memory()
        with torch.cuda.stream(stream):
            flush.zero_()
        stream.synchronize()
        t0 = time.perf_counter()
        f.insert(ins_h)
        f.erase(era_h)
        with torch.cuda.stream(stream):
            gi, gd = f.knn(q_h.to(dev, non_blocking=True), a.k)
            oi_h.copy_(gi, non_blocking=True)
            od_h.copy_(gd, non_blocking=True)
        stream.synchronize()
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
        h2d = ins.nbytes + era.nbytes + q.nbytes
        d2h = oi_h.numel() * 4 + od_h.numel() * 8 + 4 * a.batch
    f.close()

    ops_per_step = 2 * a.batch + a.queries
    res = {
        "ms": ms, "launches": launches, "prof": prof, "clocks": clk, "wall": wall,
        "knn_stats": (nodes, points, nq), "e2e_ms": statistics.median(e2e_ms) if e2e_ms else None,
        "h2d": h2d, "d2h": d2h, "ops_per_step": ops_per_step,
    }
    return res


def recorded_traffic(kernel):
    """DRAM bytes per launch of `kernel` from its committed ncu summary, or None
    when the summary is missing or the kernel source changed since the capture."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "%s_3d_10M.md" % kernel)
    try:
        text = open(path).read()
    except OSError:
        return None
    fields = dict(line.split(": ", 1) for line in text.splitlines()
                  if line.startswith(("kernel_source:", "source_sha256_16:", "dram_bytes_per_launch:")))
    try:
        src = open(os.path.join(ROOT, fields["kernel_source"].strip()), "rb").read()
    except (KeyError, OSError):
        return None
    if hashlib.sha256(src).hexdigest()[:16] != fields.get("source_sha256_16", "").strip():
        return None
    return int(fields["dram_bytes_per_launch"])


def roofline(a, res, peaks):
    """Dominant kernel of the timed region against the measured HBM peak."""
    prof = res["prof"]
    if not prof:
        return None
    name, (tot_ms, nlaunch) = max(prof.items(), key=lambda kv: kv[1][0])
    per_launch_ms = tot_ms / nlaunch
    d, k = a.dim, a.k
    R = 4 * d + 4
    nodes, points, nq = res["knn_stats"]
    algo = None
    if name == "k_knn" and nq:
        # per query: query in, k results out, one 32-B sector per visited node,
        # one record per examined leaf point
        per_q = 4 * d + 12 * k + 32 * nodes / nq + R * points / nq
        algo = per_q * a.queries
    peak = peaks.get("hbm_gbs")
    if algo is None or not peak:
        return {"kernel": name, "bound": "hbm", "achieved": None, "peak": peak, "unit": "GB/s",
                "frac": None, "traffic": None, "ms_per_launch": per_launch_ms}
    achieved = algo / (per_launch_ms * 1e-3) / 1e9
    traffic = recorded_traffic(name) if a.n0 == 10_000_000 and a.queries == 1_000_000 else None
    return {"kernel": name, "bound": "hbm", "achieved": round(achieved, 1), "peak": peak,
            "unit": "GB/s", "frac": round(achieved / peak, 4), "traffic": traffic,
            "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)" if "when" in peaks else "fallback",
            "ms_per_launch": round(per_launch_ms, 4),
            "algorithmic_bytes_per_launch": int(algo),
            "knn_visits_per_query": {"nodes": round(nodes / nq, 2), "leaf_points": round(points / nq, 2)}}


# ---------------------------------------------------------------------------
# CPU oracle (reference arm and cpu_baseline)
# ---------------------------------------------------------------------------

def oracle_sample(a, nsteps, seed=2):
    """Time the oracle on a 1/10-scale step: forest of n0/10 points, then per
    step insert batch/10, erase batch/10, k-NN for queries/10."""
    from oracle.oracle import OracleForest
    n0, b, m = a.n0 // 10, a.batch // 10, a.queries // 10
    W = StepInputs(n0, b, m, a.dim, nsteps, seed=seed)
    o = OracleForest(a.dim, leaf_size=a.leaf, buffer_size=1024)
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
    return times, ops, sample


def run_reference(a, rank):
    if rank != 0:
        return
    W = a.warmup
    times, ops, sample = oracle_sample(a, W + a.steps)
    t = times[W:]
    ms = 1e3 * sum(t) / len(t)
    value = ops / (ms * 1e-3)
    out = {"impl": "reference", "metric": METRIC, "value": round(value, 1), "unit": "ops/s",
           "n_gpus": a.gpus, "steps": a.steps, "warmup": a.warmup, "ms_per_step": round(ms, 3),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
           "data": "synthetic", "config": workload_config(a, a.gpus),
           "cpu_baseline": {"value": round(value, 1), "unit": "ops/s", "cores": 1, "kind": "oracle",
                            "sample": sample},
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
        "roofline": roofline(a, res, peaks),
        "clocks": res["clocks"],
    }
    if res["e2e_ms"]:
        out["e2e"] = {"value": round(ops / (res["e2e_ms"] * 1e-3), 1), "unit": "ops/s",
                      "h2d_bytes_per_step": res["h2d"], "d2h_bytes_per_step": res["d2h"],
                      "ms_per_step": round(res["e2e_ms"], 3)}
    if world == 1 and not a.no_cpu_baseline:
        times, ops_c, sample = oracle_sample(a, 2)
        v = ops_c / (sum(times) / len(times))
        out["cpu_baseline"] = {"value": round(v, 1), "unit": "ops/s", "cores": 1, "kind": "oracle",
                               "sample": sample}
    print(json.dumps(out), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
