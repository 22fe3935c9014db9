"""The replica path of bench.py on CPU: two gloo ranks with different timed regions agree on the
slowest rank's time and on the whole-job rate N x K / max time; the reference arm prints on rank 0 only."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms, value = bench.aggregate_replicas(100.0 + 50.0 * rank, 40, world, "cpu")
        out[rank] = (ms, value)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_slowest_time():
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    assert set(res) == {0, 1}
    for ms, value in res.values():
        assert ms == pytest.approx(150.0)
        assert value == pytest.approx(world * 40 / 0.150)


def test_single_rank_needs_no_process_group():
    import bench
    ms, value = bench.aggregate_replicas(80.0, 20, 1)
    assert ms == 80.0 and value == pytest.approx(20 / 0.080)


def test_reference_arm_prints_on_rank_zero_only(monkeypatch, capsys):
    import bench

    class A:
        workload, steps, warmup, gpus = "img64_m2k", 1, 0, 2
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    bench.run_reference(A())
    assert capsys.readouterr().out == ""
