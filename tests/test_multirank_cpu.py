"""The N > 1 path of bench.py on CPU: two gloo ranks run the replica bookkeeping
(barrier, max over ranks of the timed region, whole-job rate) that the GPU
ranks run under torchrun. No GPU: each rank stands in a fixed elapsed time."""

import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        bench.barrier(world)
        elapsed = 1.0 + rank  # rank 1 is the slow one
        t = bench.max_over_ranks(elapsed, world, "cpu")
        out[rank] = (t, bench.whole_job_rate(1000.0, t, world))
        bench.barrier(world)
    finally:
        dist.destroy_process_group()


def test_two_rank_replica_bookkeeping():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank, args=(world, _free_port(), out), nprocs=world, start_method="spawn", join=True)
    assert out[0] == out[1]
    t, rate = out[0]
    assert t == 2.0  # max over ranks
    assert rate == pytest.approx(world * 1000.0 / 2.0)
