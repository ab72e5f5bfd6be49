"""The N-GPU benchmark path on CPU ranks (gloo, world size 2).

Every rank owns an independent forest (the path shards into independent
problems), so the only cross-rank steps are the barrier and the maximum of
the per-phase times; rank 0 reports the whole job's rate.  Here two CPU ranks
stand in for two GPUs."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = {"step": 10.0 + rank, "insert": 3.0 - rank, "erase": 2.0, "knn": 5.0 + 2 * rank}
    dist.barrier()
    cpu = torch.device("cpu")
    out = bench.max_over_ranks(ms, dist, cpu)
    leaf = bench.rank0_choice(16 + 8 * rank, dist, cpu)     # each rank tuned its own
    e2e = bench.slowest(6.0 + 0.5 * rank, dist, cpu)
    q.put((rank, out, bench.job_throughput(3_000_000, world, out["step"]), leaf, e2e))
    dist.destroy_process_group()


def test_two_ranks_take_the_slowest_phase_times():
    """Phase and end-to-end times are the slowest rank's; an autotuned leaf
    size is rank 0's on every rank."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for rank, ms, rate, leaf, e2e in got:
        assert ms == {"step": 11.0, "insert": 3.0, "erase": 2.0, "knn": 7.0}
        assert rate == pytest.approx(3_000_000 * 2 / 11e-3)
        assert leaf == 16           # rank 0's tuned leaf size on every rank
        assert e2e == 6.5           # the slowest rank's end-to-end step


def test_reference_arm_other_ranks_exit_quietly(capsys):
    import bench
    args = type("A", (), {})()
    bench.run_reference(args, rank=1)     # rank != 0: no work, no output
    assert capsys.readouterr().out == ""
