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


def _serve_worker(rank, world, port, out):
    """Each rank draws its own request stream (bench.serve_seed) and solves
    the first requests that the oracle finishes quickly; the ranks exchange
    only their results' checksums, after the work (no data-path collective)."""
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    out[rank] = _solve_own_stream(rank)
    got = [None] * world
    dist.all_gather_object(got, out[rank])
    assert got[rank] == out[rank]
    dist.destroy_process_group()


def _solve_own_stream(rank, count=2, max_nodes=7000):
    import numpy as np
    import bench
    from oracle.smpm import Grid
    from oracle import dbj
    from paper_1512_01756_gb300 import inputs
    reqs = [q for q in bench.serve_stream(60, bench.serve_seed(rank))
            if (q["order"] + 1) ** 2 * q["mx"] * q["mz"] <= max_nodes][:count]
    res = []
    for q in reqs:
        lx = q["mx"] / q["mz"]
        g = Grid(q["mx"], q["mz"], q["order"], lx, 1.0)
        X, Z = g.coords()
        f, _ = inputs.cos_modes(X, Z, lx, 1.0, inputs.cos_modes_spec(q["seed"]))
        u, info = dbj.solve(g, f, k2=q["k2"], method="dbj", tol=1e-12)
        res.append((q["seed"], q["mx"], q["mz"], q["order"], q["k2"], float(np.sum(u * u)), info["schur_residual"]))
    return res


def test_two_gloo_ranks_serve_their_own_streams():
    """The serving bench's partition: rank r's requests and results are those
    a single process computes for rank r's stream (they do not depend on the
    world size), the two ranks' requests are disjoint, and every oracle solve
    meets its tolerance."""
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.start_processes(_serve_worker, args=(world, port, out), nprocs=world, start_method="spawn", join=True)
        res = dict(out)
    seeds = [set(r[0] for r in res[k]) for k in range(world)]
    assert not seeds[0] & seeds[1]
    for rank in range(world):
        alone = _solve_own_stream(rank)
        assert len(res[rank]) == len(alone) == 2
        for a, b in zip(res[rank], alone):
            assert a[:5] == b[:5]
            assert abs(a[5] - b[5]) <= 1e-12 * abs(b[5])
            assert a[6] < 1e-11
