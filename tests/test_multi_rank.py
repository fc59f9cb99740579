"""Host logic of the N-GPU bench (one process per GPU, weak scaling): each
rank parses its own independently seeded shard, the job time is the
slowest rank's, and the whole-job value counts every rank's bytes.  Run
here as two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench
from paper_2101_11408_gb300 import workloads


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = [12.5, 40.0][rank]            # rank 1 is the slow one
        job_ms = bench.max_over_ranks(dist, ms, torch.device("cpu"))
        text = workloads.uniform_text(200, bench.shard_seed(workloads.SEED_BASE + 1, rank))
        dist.barrier()
        q.put((rank, job_ms, len(text), hash(text)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time_and_distinct_shards():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [40.0, 40.0]
    assert res[0][3] != res[1][3]          # independent shards
    total = sum(r[2] for r in res)
    # whole-job GB/s: every rank's bytes over the slowest rank's time
    per_rank = res[0][2]
    assert bench.whole_job_gbs(world, per_rank, 10, 40.0) == pytest.approx(
        world * per_rank * 10 / 0.040 / 1e9)
    assert total > 0


def test_single_process_needs_no_collective():
    assert bench.max_over_ranks(None, 3.5, None) == 3.5
    assert bench.whole_job_gbs(1, 10**9, 1, 1000.0) == pytest.approx(1.0)
