"""The multi-rank path of bench.py on CPU ranks (gloo, world size 2):
whole-job throughput = all ranks' units over the slowest rank's time."""
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


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t_ms = [100.0, 250.0][rank]          # rank 1 is the slowest
    units = [2000, 2000][rank]
    value, t_max = bench.aggregate(t_ms, units, world)
    out[rank] = (value, t_max)
    dist.destroy_process_group()


def test_aggregate_max_over_ranks():
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(2, _free_port(), out), nprocs=2, join=True)
    for r in range(2):
        value, t_max = out[r]
        assert t_max == 250.0
        assert abs(value - 4000 / 0.25) < 1e-6
