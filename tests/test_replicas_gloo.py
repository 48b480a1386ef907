"""The multi-process path of the benchmark on CPU: each rank is an
independent replica (no collective on the data path); the whole-job value is
the matvecs of all ranks over the slowest rank's time. Two gloo ranks."""
import os
import socket
import sys

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    assert bench.dist_env() == (world, rank, rank)
    # rank r ran 48 * (r + 1) matvecs in 1000 * (r + 1) ms
    value, total_ms, matvecs = bench.aggregate_replicas(dist, 1000.0 * (rank + 1), 48 * (rank + 1), "cpu")
    out[rank] = (value, total_ms, matvecs)
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_aggregate_max_time_sum_work():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, out), nprocs=2, join=True, start_method="spawn")
    for r in range(2):
        value, total_ms, matvecs = out[r]
        assert total_ms == 2000.0          # the slowest rank's time
        assert matvecs == 48 + 96          # all ranks' work
        assert value == pytest.approx(144 / 2.0)


def test_single_process_is_unchanged():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate_replicas(None, 500.0, 16, "cpu") == (32.0, 500.0, 16)
