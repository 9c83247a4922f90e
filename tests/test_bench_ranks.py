"""The N > 1 path of bench.py without a GPU: every rank renders its own replica
(the render has no cross-GPU exchange), and the job's time is the slowest
rank's. Two gloo ranks on 127.0.0.1 check the max-over-ranks reduction and the
whole-job throughput; the reference arm does its work on rank 0 only."""
import os
import socket

import pytest

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, local_ms, out):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = bench.slowest_rank(local_ms[rank], world)
        out[rank] = (ms, bench.job_throughput(960 * 540 * 10, world, ms * 1e-3))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    import torch.multiprocessing as mp

    world, port = 2, _free_port()
    local_ms = [3.5, 5.25]
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(world, port, local_ms, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0] == res[1]
    ms, value = res[0]
    assert ms == max(local_ms)
    assert value == pytest.approx(960 * 540 * 10 * world / (max(local_ms) * 1e-3) / 1e6)


def test_single_rank_is_identity():
    assert bench.slowest_rank(7.0, 1) == 7.0
    assert bench.job_throughput(1_000_000, 1, 0.5) == pytest.approx(2.0)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class Args:
        workload, steps, warmup = "tiny", 1, 1

    assert bench.run_reference(Args()) is None
    assert capsys.readouterr().out == ""
