"""The multi-GPU path is replicas only: every rank runs the whole workload
on its own GPU, with no collective on the data path; the ranks meet only to
time the job.  These world-size-2 gloo tests run that host logic on CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp

from conftest import ROOT


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import sys
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    # each rank reports its own timings; the slowest bounds the job
    got = bench.reduce_max([1.0 + rank, 10.0 * (world - rank)], "cpu")
    value = bench.whole_job_value(5e9, world, got[0])
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, got, value))


@pytest.mark.parametrize("world", [2])
def test_reduce_max_and_whole_job_value_over_gloo(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, got, value in out:
        assert got == [float(world), 10.0 * world]
        assert abs(value - world * 5.0 / world) < 1e-12  # 2 ranks x 5e9 units / 2 s


def test_single_rank_needs_no_process_group():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_max([3.0, 4.0], "cpu") == [3.0, 4.0]
    assert bench.whole_job_value(6e9, 1, 2.0) == 3.0
