"""Host logic of bench.py's multi-rank path, on CPU with the gloo backend and
world size 2: each rank's right-hand sides are its own (disjoint seeds), the
job's time is the maximum over ranks and every rank sees it, and the
reference arm runs on rank 0 only (other ranks exit without work)."""
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
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    seeds = [bench.rank_seed0(rank) + i for i in range(16)]
    got = [None] * world
    dist.all_gather_object(got, seeds)
    t = bench.max_over_ranks(10.0 + rank, torch.device("cpu"), world)
    out[rank] = (t, got)
    dist.destroy_process_group()


def test_two_gloo_ranks_partition_and_max():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.start_processes(_worker, args=(world, port, out), nprocs=world, start_method="spawn", join=True)
        res = dict(out)
    for rank in range(world):
        t, seeds = res[rank]
        assert t == 11.0                                  # the slowest rank's time, on every rank
        assert not set(seeds[0]) & set(seeds[1])          # disjoint right-hand sides
        assert len(seeds[0]) == len(set(seeds[0])) == 16


def test_reference_arm_runs_on_rank0_only(monkeypatch, capsys):
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    assert bench.run_reference(None) == 0                 # returns before reading its arguments
    assert capsys.readouterr().out == ""
