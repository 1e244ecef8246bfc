"""The multi-GPU path of bench.py is replicas only: every rank solves its own
copy, the job time is the slowest rank's and the work the sum over ranks.
Checked with two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    times = [10.0 + rank, 5.0 * (rank + 1), 7.0]
    counts = [100 * (rank + 1), 3, 0.5]
    t, c = bench.reduce_over_ranks(dist, times, counts, "cpu")
    out[rank] = (t, c)
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_max_time_sum_work():
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        t, c = res[rank]
        assert t == [11.0, 10.0, 7.0]
        assert c == [300.0, 6.0, 1.0]


def test_dist_env_defaults_to_one_rank(monkeypatch):
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    assert bench.dist_env() == (0, 1, 0)
