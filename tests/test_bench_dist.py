"""Host-side logic of bench.py's multi-rank path, on CPU with gloo (no GPU):
independent replicas, max-over-ranks time, whole-job throughput; and the
reference arm running on rank 0 only."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    tmax, rate = bench.aggregate(10.0 * (rank + 1), 1000.0, dist, "cpu")
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, tmax, rate))


def test_aggregate_two_ranks_gloo():
    import socket

    import torch.multiprocessing as mp
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, tmax, rate in out:
        assert tmax == pytest.approx(20.0)               # the slowest rank
        assert rate == pytest.approx(2 * 1000.0 / 0.020)  # all ranks' units


def test_aggregate_single_rank():
    sys.path.insert(0, ROOT)
    import bench
    tmax, rate = bench.aggregate(5.0, 100.0)
    assert tmax == 5.0 and rate == pytest.approx(100.0 / 0.005)


def test_reference_arm_only_on_rank_zero(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import argparse

    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    args = argparse.Namespace(gpus=2, steps=1, warmup=3, ref_sample_steps=1)
    assert bench.run_reference(args) == 0
    assert capsys.readouterr().out == ""
