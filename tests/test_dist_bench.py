"""The N > 1 aggregation of bench.py on two CPU processes (gloo): every rank sees the
slowest rank's time, and the job throughput counts the nodes of all replicas."""
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


def _worker(rank, world, port, times, out):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w, r, _ = bench.dist_env()
    total = bench.max_over_ranks(times[rank])
    out[rank] = (w, r, total, bench.job_mlups(w, 1000, 10, total))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_aggregation():
    world, port = 2, _free_port()
    times = [12.5, 20.0]
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, port, times, out), nprocs=world, join=True, start_method="spawn")
    assert sorted(out.keys()) == [0, 1]
    for rank in range(world):
        w, r, total, value = out[rank]
        assert (w, r) == (2, rank)
        assert total == 20.0                                  # the slowest rank
        assert abs(value - 2 * 1000 * 10 / 20e-3 / 1e6) < 1e-12   # both replicas' nodes


def test_single_process_passthrough():
    import bench
    assert bench.max_over_ranks(3.25) == 3.25
    assert bench.job_mlups(1, 10**6, 100, 1000.0) == 100.0
