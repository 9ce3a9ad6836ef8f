"""bench.py at N > 1 runs independent replicas: each rank times its own
stream, and the job's figure is all ranks' edges over the slowest rank's
time.  The reduction is checked here with two gloo ranks on the CPU."""
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
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t, units = bench.reduce_over_ranks(dist, 10.0 + 5.0 * rank, 1000 * (rank + 1), "cpu")
    dist.barrier()
    out[rank] = (t, units)
    dist.destroy_process_group()


def test_replicas_take_max_time_and_sum_units():
    world = 2
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        assert res[r] == (15.0, 3000.0)


def test_single_process_is_unchanged():
    import bench
    assert bench.reduce_over_ranks(None, 2.5, 7, "cpu") == (2.5, 7.0)
