"""Multi-rank host logic of bench.py on the CPU: world-size-2 gloo ranks
(replicas, no data-path collective) agree on the slowest rank's step time,
the reported value counts every rank's work, and the reference arm's other
ranks leave without work."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, times, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = bench.rank_max(times[rank], dist, torch.device("cpu"))
        value = bench.whole_job_rate(300, world, ms)
        out[rank] = (ms, value)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_step():
    world, times = 2, [210.0, 250.0]
    port = _free_port()
    out = mp.get_context("spawn").Manager().dict()
    mp.start_processes(_rank_main, args=(world, port, times, out), nprocs=world, join=True, start_method="spawn")
    assert out[0] == out[1]
    ms, value = out[0]
    assert ms == max(times)
    assert value == pytest.approx(300 * world / (max(times) / 1e3))


def test_single_rank_keeps_its_own_time():
    assert bench.rank_max(123.5, None, None) == 123.5
    assert bench.whole_job_rate(300, 1, 250.0) == pytest.approx(1200.0)


def test_reference_arm_other_ranks_do_no_work(capsys):
    class Args:
        gpus, steps, warmup = 2, 1, 0
    assert bench.run_reference(Args(), rank=1) == 0
    assert capsys.readouterr().out == ""
