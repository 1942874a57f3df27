"""bench.py's multi-rank logic on CPU: world_size 2 over gloo.

Under torchrun every rank advances its own replica; the timed region is the
maximum over ranks and the rate is that of all replicas together. These
tests run the same helpers bench.py uses, with two gloo ranks on 127.0.0.1,
and check the rank handling of the launcher environment and of the
reference arm (rank 0 alone does the work).
"""

import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w, r, lr = bench.dist_setup(world)
    assert (w, r, lr) == (world, rank, rank)
    elapsed = 1.0 + rank                   # rank 1 is the slow one
    dist.barrier()
    slowest = bench.max_over_ranks(elapsed, dist, "cpu")
    out[rank] = (slowest, bench.whole_job_rate(world, 1000, 10, slowest))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    world, port = 2, _free_port()
    out = mp.Manager().dict()
    mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
    assert out[0] == out[1] == (2.0, 2 * 1000 * 10 / 2.0 / 1e9)


def test_launcher_environment(monkeypatch):
    import bench

    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("LOCAL_RANK", "1")
    assert bench.dist_setup(2) == (2, 1, 1)
    with pytest.raises(SystemExit):
        bench.dist_setup(4)                # --gpus disagrees with the launcher
    monkeypatch.setenv("WORLD_SIZE", "1")
    monkeypatch.setenv("RANK", "0")
    monkeypatch.setenv("LOCAL_RANK", "0")
    assert bench.dist_setup(1) == (1, 0, 0)
    assert bench.max_over_ranks(3.5, None, "cpu") == 3.5


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    import bench

    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("LOCAL_RANK", "1")
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--gpus", "2"])
    bench.main()                           # returns at once: no oracle work, no output
    assert capsys.readouterr().out == ""
