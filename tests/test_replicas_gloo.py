"""The multi-GPU mode of the benchmark is replicas only: every rank evaluates its
own copy of the workload, with no collective in the data path; the ranks only
agree on the job's time (the slowest rank's) and rank 0 reports the whole-job
rate.  Checked here with two gloo ranks on the CPU."""
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank: int, world: int, port: int, q):
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    try:
        own_ms = [120.0, 250.0][rank]              # rank 1 is the slow replica
        dist.barrier()
        total = bench.reduce_max(own_ms, torch.device("cpu"), world)
        rate = bench.whole_job_rate(1_000_000, 10, total, world)
        q.put((rank, total, rate))
    finally:
        dist.destroy_process_group()


def test_reduce_max_and_rate_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    got = sorted(q.get(timeout=5) for _ in range(2))
    for rank, total, rate in got:
        assert total == 250.0                       # both ranks see the slowest time
        # 2 replicas x 1e6 particles x 10 steps in 0.25 s
        assert rate == pytest.approx(2 * 1e6 * 10 / 0.25 / 1e6)


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_max(3.5, torch.device("cpu"), 1) == 3.5
    assert bench.whole_job_rate(2_097_152, 60, 600.0, 1) == pytest.approx(2_097_152 * 60 / 0.6 / 1e6)
