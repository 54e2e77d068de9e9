"""The multi-GPU path of the bench is replicas only (one independent instance
per rank, no collective on the data path): two gloo ranks on the CPU check
its only collective (the slowest rank's times) and the whole-job value, and
that the reference arm does its work on rank 0 alone."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r "took" (1 + r, 2 + 3 r, 0.5) seconds for the three arms
        mine = [1.0 + rank, 2.0 + 3.0 * rank, 0.5]
        slow = bench.slowest_rank(dist, torch, "cpu", mine)
        dist.barrier()
        out[rank] = slow
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_replica():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0] == res[1] == [2.0, 5.0, 0.5]
    # 10 steps on each of 2 replicas, the slower one taking 2 s: 10 steps/s for the job
    assert bench.replica_value(world, 10, res[0][0]) == pytest.approx(10.0)


def test_single_process_needs_no_collective():
    assert bench.slowest_rank(None, torch, "cpu", [1.5, 2.5]) == [1.5, 2.5]


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class Args:
        steps, warmup, cpu_budget = 1, 0, 1.0

    bench.run_reference(Args())     # returns at once: no oracle run, no output
    assert capsys.readouterr().out == ""
