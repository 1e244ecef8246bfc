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


def _ref_worker(rank, world, port, outdir):
    import contextlib
    import json as _json
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    args = bench.parse(["--impl", "reference", "--gpus", str(world), "--steps", "2", "--warmup", "1",
                             "--n", "12"])
    path = os.path.join(outdir, f"rank{rank}.out")
    with open(path, "w") as f, contextlib.redirect_stdout(f):
        bench.run_reference(args)
    lines = [l for l in open(path) if l.strip()]
    if lines:
        _json.loads(lines[0])


def test_reference_arm_two_ranks_rank0_prints_one_line(tmp_path):
    """Under two ranks the reference arm (the oracle on the host) runs and
    prints on rank 0 only; rank 1 exits without work."""
    import json
    world = 2
    mp.spawn(_ref_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    out0 = [l for l in open(tmp_path / "rank0.out") if l.strip()]
    out1 = [l for l in open(tmp_path / "rank1.out") if l.strip()]
    assert len(out0) == 1 and out1 == []
    line = json.loads(out0[0])
    assert line["impl"] == "reference" and line["unit"] == "MLUP/s" and line["value"] > 0
    assert line["steps"] == 2 and line["warmup"] == 1 and line["n_gpus"] == 2
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0


def test_traffic_counters_scale_with_cells_and_expire_with_the_sources(monkeypatch):
    """The committed DRAM counters are per captured cell, taken on the current
    sweep sources; a changed source hash makes them unavailable (null)."""
    import json
    d = json.load(open(os.path.join(bench.ROOT, "profiles", "traffic.json")))
    current = d["src_hash"] == bench.src_hash()
    for kernel, v in d["kernels"].items():
        assert kernel in bench.ALGO_BYTES
        per_cell = v["captured_bytes"] / v["captured_cells"]
        # DRAM traffic within the algorithmic bytes plus the records' pad words
        assert 0.5 * bench.ALGO_BYTES[kernel] <= per_cell <= 1.25 * bench.ALGO_BYTES[kernel], kernel
        if current:
            assert bench.load_traffic(kernel, 1000) == round(per_cell * 1000)
            assert bench.load_traffic(kernel, 2000) == round(per_cell * 2000)
        else:  # counters of other sources are never reported
            assert bench.load_traffic(kernel, 1000) is None
    monkeypatch.setattr(bench, "src_hash", lambda: "0" * 16)
    assert bench.load_traffic("fwd32", 1000) is None
