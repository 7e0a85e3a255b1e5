"""The benchmark's multi-rank protocol on CPU (gloo, world size 2): every
rank takes the slowest rank's clock, the whole-job rate counts the units of
all ranks, and only rank 0 of the oracle arm does work and reports."""
import os
import socket
import types

import torch
import torch.multiprocessing as mp

import bench


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        reduce_max = bench.max_over_ranks_fn(dist, torch.device("cpu"))
        local_ms = 100.0 * (rank + 1)  # rank 1 is the slow one
        slowest = reduce_max(local_ms)
        dist.barrier()
        q.put((rank, slowest, bench.whole_job_rate(5, slowest, world)))
    finally:
        dist.destroy_process_group()


def test_two_ranks_report_the_slowest_clock():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [g[0] for g in got] == [0, 1]
    for _, slowest, rate in got:
        assert slowest == 200.0
        assert rate == 2 * 5 / 0.2  # ten reconstructions in the slowest rank's 0.2 s


def test_single_rank_is_the_identity():
    assert bench.max_over_ranks_fn(None, None)(12.5) == 12.5
    assert bench.whole_job_rate(3, 1500.0, 1) == 2.0


def test_reference_arm_runs_on_rank_zero_only():
    args = types.SimpleNamespace(workload="n128", steps=1, warmup=0)
    assert bench.run_reference(args, rank=1) is None
