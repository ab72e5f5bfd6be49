"""Autotuner: leaf size, and the k-NN kernel's block size and queries per warp.

The leaf size L (points per leaf, Sec. V-D) trades tree height -- node
visits per query and levels per build -- against points scanned per leaf.
The k-NN answers do not depend on it (they are the exact k nearest by
(squared distance, id)), only the speed does, so L can be chosen per
workload by measurement: for every candidate, build a forest on the
workload's own initial points and time a few steps of it (one insert batch,
one erase batch, one k-NN batch) with CUDA events; the fastest mean step
wins, except that the default leaf size is kept unless another candidate is
faster by more than TIE (step times of neighbouring leaf sizes are often
within the noise of a few steps).

The k-NN launch shape (threads per block, queries per warp) changes neither
the trees nor the answers, only the k-NN kernel's speed, so it is tuned
after L on one forest of the chosen L: the tuning steps' updates are applied,
then every shape answers the same query batches, in round-robin order over
the shapes so that drift hits them alike; the fastest mean k-NN time wins,
with the same tie rule towards the default shape.  Every step runs in the
CUDA library; this module only times calls.
"""
import numpy as np
import torch

from . import inputs
from .forest import Forest

CANDIDATES = (8, 12, 16, 24, 32)
CONFIG_CANDIDATES = (8, 16, 32)   # the leaf sizes the 10M-point 3-D workload names
DEFAULT = 16
TIE = 0.01
# k-NN launch shapes (threads per block, queries per warp)
SHAPES = tuple((b, q) for b in (64, 128, 256) for q in (32, 64, 128))
DEFAULT_SHAPE = (128, 32)


def choose(ms, default=DEFAULT):
    """The candidate to use given {candidate: mean ms}: the fastest, unless
    the default is within TIE of it."""
    best = min(ms, key=ms.get)
    if default in ms and ms[best] > ms[default] * (1.0 - TIE):
        return default
    return best


def _time_shapes(forests, run_knn, queries, shapes, reps, stream):
    """{shape: mean ms of one k-NN call}: every shape answers every query
    batch `reps` times, shapes interleaved; run_knn(q) issues one call."""
    L2 = torch.empty(256 << 20, dtype=torch.uint8, device=stream.device)
    times = {sh: [] for sh in shapes}
    for f in forests:                        # one untimed call per shape
        f.set_knn_shape(*shapes[0])
    run_knn(queries[0])
    for r in range(reps + 1):
        for q in queries:
            for sh in shapes:
                for f in forests:
                    f.set_knn_shape(*sh)
                with torch.cuda.stream(stream):
                    L2.zero_()               # no query batch starts with a warm L2
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(stream)
                run_knn(q)
                b.record(stream)
                b.synchronize()
                if r:                        # the first round warms every shape up
                    times[sh].append(a.elapsed_time(b))
    for f in forests:
        f.set_knn_shape(*DEFAULT_SHAPE)
    return {sh: float(np.mean(v)) for sh, v in times.items()}


def tune_knn_shape(dim, leaf, initial, steps, k, shapes=SHAPES, reps=2, device=None, stream=None,
                   split="object"):
    """The fastest k-NN launch shape (block threads, queries per warp) for a
    forest of leaf size `leaf` after the updates of `steps` (device-tensor
    triples as in tune_leaf_size), timed on the steps' query batches; and the
    mean k-NN ms of each shape."""
    stream = stream or torch.cuda.current_stream(device)
    f = Forest(dim, leaf_size=leaf, stream=stream, device=device, split=split)
    try:
        f.insert(initial)
        for ins, era, _ in steps:
            f.insert(ins)
            f.erase(era)
        ms = _time_shapes([f], lambda q: f.knn(q, k), [q for _, _, q in steps], list(shapes), reps, stream)
        return choose(ms, DEFAULT_SHAPE), ms
    finally:
        f.close()


def time_steps(dim, leaf, initial, steps, k, device=None, stream=None, split="object"):
    """Mean milliseconds of one (insert, erase, k-NN) step over `steps`, on a
    forest of `initial` (device tensor) with leaf size `leaf`; the first step
    is a warm-up and is not counted."""
    stream = stream or torch.cuda.current_stream(device)
    f = Forest(dim, leaf_size=leaf, stream=stream, device=device, split=split)
    try:
        f.insert(initial)
        times = []
        for i, (ins, era, q) in enumerate(steps):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            f.insert(ins)
            f.erase(era)
            f.knn(q, k)
            b.record(stream)
            b.synchronize()
            if i:
                times.append(a.elapsed_time(b))
        return float(np.mean(times))
    finally:
        f.close()


def tune_leaf_size(dim, initial, steps, k, candidates=CANDIDATES, device=None, stream=None, split="object"):
    """The fastest leaf size among `candidates` for this workload, and the
    measured mean step time (ms) of each.  `initial` is a device tensor of
    points; `steps` a list of at least two (insert points, erase ids, queries)
    device-tensor triples."""
    if len(steps) < 2:
        raise ValueError("need a warm-up step and at least one timed step")
    ms = {L: time_steps(dim, L, initial, steps, k, device, stream, split) for L in candidates}
    return choose(ms), ms


def synthetic_steps(dim, n0, batch, queries, nsteps, seed, device=None):
    """A uniform forest of n0 points and `nsteps` steps of the shape the
    autotuner times (insert `batch`, erase `batch` live ids, `queries`
    live-set queries), all on the device."""
    dev = device or torch.device("cuda")
    pts = inputs.uniform_points(n0, dim, seed)
    live = inputs.LiveSet(dim)
    live.insert(pts)
    rng = np.random.default_rng(seed + 1)
    steps = []
    for _ in range(nsteps):
        ins = rng.integers(0, inputs.GRID, size=(batch, dim), dtype=np.int32)
        live.insert(ins)
        era = rng.choice(live.live_ids(), size=min(batch, int(live.alive.sum())), replace=False)
        live.erase(era)
        lid = live.live_ids()
        q = live.coords[lid[rng.integers(0, len(lid), size=queries)]]
        T = lambda x: torch.from_numpy(np.ascontiguousarray(x)).to(dev)
        steps.append((T(ins), T(era.astype(np.int32)), T(q)))
    return torch.from_numpy(pts).to(dev), steps


def time_forests_step(dims, leaf, initial, steps, k, device=None, stream=None, split="object"):
    """Mean milliseconds of one batched step (insert, erase, k-NN over all the
    forests in one call each) for forests with leaf size `leaf`; `initial[i]`
    is forest i's first points and every step a list of per-forest (insert
    points, erase ids, queries), all device tensors.  The first step is a
    warm-up."""
    from .forest import erase_batch, insert_batch, knn_batch
    stream = stream or torch.cuda.current_stream(device)
    forests = [Forest(d, leaf_size=leaf, stream=stream, device=device, split=split) for d in dims]
    try:
        insert_batch(forests, initial, stream=stream)
        times = []
        for i, st in enumerate(steps):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            insert_batch(forests, [x for x, _, _ in st], stream=stream)
            erase_batch(forests, [e for _, e, _ in st], stream=stream)
            knn_batch(forests, [q for _, _, q in st], k, stream=stream)
            b.record(stream)
            b.synchronize()
            if i:
                times.append(a.elapsed_time(b))
        return float(np.mean(times))
    finally:
        for f in forests:
            f.close()


def tune_knn_shape_forests(dims, leaf, initial, steps, k, shapes=SHAPES, reps=2, device=None, stream=None,
                           split="object"):
    """tune_knn_shape for a batched many-forest workload: the forests take
    the steps' updates in batched calls, then every shape answers the steps'
    batched query sets (the batched call launches with the first forest's
    shape; every forest gets the same)."""
    from .forest import erase_batch, insert_batch, knn_batch
    stream = stream or torch.cuda.current_stream(device)
    forests = [Forest(d, leaf_size=leaf, stream=stream, device=device, split=split) for d in dims]
    try:
        insert_batch(forests, initial, stream=stream)
        for st in steps:
            insert_batch(forests, [x for x, _, _ in st], stream=stream)
            erase_batch(forests, [e for _, e, _ in st], stream=stream)
        ms = _time_shapes(forests, lambda qs: knn_batch(forests, qs, k, stream=stream),
                          [[q for _, _, q in st] for st in steps], list(shapes), reps, stream)
        return choose(ms, DEFAULT_SHAPE), ms
    finally:
        for f in forests:
            f.close()


def tune_leaf_size_forests(dims, initial, steps, k, candidates=CANDIDATES, device=None, stream=None,
                           split="object"):
    """The fastest leaf size among `candidates` for a batched many-forest
    workload (one leaf size for all forests), and each candidate's mean step
    time (ms)."""
    if len(steps) < 2:
        raise ValueError("need a warm-up step and at least one timed step")
    ms = {L: time_forests_step(dims, L, initial, steps, k, device, stream, split) for L in candidates}
    return choose(ms), ms
