"""Multi-rank host logic of bench.py on the CPU (gloo, two ranks): every rank works on
its own units, the whole-job rate is the units of all ranks over the slowest rank's
time, and under a launcher only rank 0 runs the reference arm."""
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    dist.init_process_group("gloo", init_method="env://", rank=rank, world_size=world)
    try:
        w, r, lr = bench.rank_env()
        elapsed = 2.0 if rank == 1 else 1.0           # rank 1 is the slow one
        dist.barrier()
        tmax, value = bench.whole_job_rate(elapsed, 300, torch.device("cpu"))
        q.put((rank, w, r, lr, bench.unit_seed(7, rank), tmax, value))
    finally:
        dist.destroy_process_group()


def test_two_ranks_gloo():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(world))
    seeds = {g[4] for g in got}
    assert seeds == {7, 8}                            # independent units per rank
    for rank, w, r, lr, _, tmax, value in got:
        assert (w, r, lr) == (world, rank, rank)
        assert tmax == 2.0                            # the slowest rank's time
        assert value == pytest.approx(300 * world / 2.0)


def test_single_process_rate():
    tmax, value = bench.whole_job_rate(0.5, 100, torch.device("cpu"))
    assert tmax == 0.5 and value == pytest.approx(200.0)


def test_reference_arm_other_ranks_exit_quietly(capsys, monkeypatch):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--gpus", "2", "--steps", "1"])
    assert bench.main() == 0
    assert capsys.readouterr().out == ""
