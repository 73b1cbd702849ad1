"""Multi-process replicas of bench.py on the CPU (gloo, world size 2): every rank
solves its own instance and the job's time is the slowest rank's.  The GPU path
has no cross-rank data exchange, so the host logic is what the processes share."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, values, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    out[rank] = bench.max_over_ranks(values[rank], world, "cpu")
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_gloo_world2():
    port = _free_port()
    values = [3.25, 7.5]
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(2, port, values, out), nprocs=2, join=True)
        assert out[0] == out[1] == pytest.approx(7.5)


def test_max_over_ranks_single():
    import bench
    assert bench.max_over_ranks(4.0, 1, "cpu") == 4.0
