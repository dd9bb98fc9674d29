"""The multi-GPU path is replicas only (signals are independent): each rank runs the same
per-GPU batch and the job's time is the slowest rank's.  This checks that host logic with
two gloo ranks on the CPU: the MAX all-reduce of the step times and the whole-job
throughput, and that the reference arm runs on rank 0 alone."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    w, r, loc = bench._dist()
    ms_local = [20.0, 25.0][rank]                 # rank 1 is the slower one
    ms_max, value = bench.job_throughput(ms_local, 64, w, "cpu")

    class A:
        steps, warmup = 1, 0
    ref = bench.run_reference(A) if rank != 0 else "rank0"
    out[rank] = (w, r, loc, ms_max, value, ref)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
    for rank in range(world):
        w, r, loc, ms_max, value, ref = out[rank]
        assert (w, r, loc) == (world, rank, rank)
        assert ms_max == 25.0
        assert abs(value - 64 * world / 0.025) < 1e-6
    assert out[1][5] is None                      # the reference arm: rank 0 only
