"""Multi-rank logic of bench.py on CPU (gloo, world size 2): every rank runs
an independent replica, the slowest rank's time decides, and the job rate is
all ranks' particles over that time. No GPU."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = 5.0 + 2.0 * rank                      # rank 1 is slower
    slowest = bench.reduce_max(ms)
    out[rank] = (slowest, bench.job_throughput(1_000_000, world, slowest), bench._dist())
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_gloo():
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        slowest, rate, d = res[rank]
        assert slowest == 7.0                   # max over ranks
        assert abs(rate - 2 * 1_000_000 / 7.0e-3) < 1e-6 * rate
        assert d == (world, rank, rank)


def test_single_process_reduce_is_identity():
    import bench
    assert bench.reduce_max(3.5) == 3.5
    assert bench.job_throughput(10, 1, 1000.0) == 10.0


def test_reference_arm_other_ranks_exit(monkeypatch, capsys):
    """Under torchrun only rank 0 runs the CPU reference; the others exit 0."""
    import argparse

    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    args = argparse.Namespace(gpus=2, steps=1, warmup=0)
    assert bench.run_reference(args) == 0
    assert capsys.readouterr().out == ""
