"""The multi-GPU form of the benchmark on CPU: two gloo ranks (CPU only).

The path does not shard (each solve runs on one GPU), so N GPUs run N
independent replicas: the ranks meet at a barrier, the job time is the maximum
of the ranks' times and the whole-job rate is all ranks' solves over it. These
checks run that host logic (bench.Replicas) over world size 2 with gloo on
127.0.0.1; the device work of each rank is the single-GPU path.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        r = bench.Replicas(dist, "cpu")
        r.barrier()
        local = 1.5 + rank                      # this rank's timed region, seconds
        m = r.max(local)
        out.put((rank, r.world, m, r.rate(10, m)))
        r.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_replicas_max_time_and_whole_job_rate():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert [r[0] for r in res] == [0, 1]
    for _, world, m, rate in res:
        assert world == 2 and m == 2.5                 # the slower rank sets the job time
        assert rate == pytest.approx(2 * 10 / 2.5)      # all ranks' solves over that time


def test_single_process_is_one_replica():
    import bench
    r = bench.Replicas(None)
    assert r.world == 1 and r.max(3.0) == 3.0 and r.rate(10, 2.0) == 5.0
    r.barrier()
