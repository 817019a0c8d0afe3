"""The N > 1 host path of bench.py (independent replicas, one per rank): the
job time is the slowest rank's and the value is world x units / that time.
Two gloo ranks on the CPU (no GPU)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        ms = 100.0 + 50.0 * rank  # rank 1 is the slow replica
        ms_max = bench.max_over_ranks(ms, world, "cpu")
        out[rank] = (ms_max, bench.job_throughput(1000.0, ms_max / 1e3, world))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_replicas_take_the_slowest_time():
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank_main, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
    assert out[0] == out[1]
    ms_max, value = out[0]
    assert ms_max == 150.0
    assert value == pytest.approx(2 * 1000.0 / 0.150)


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(42.0, 1) == 42.0
    assert bench.job_throughput(10.0, 2.0, 1) == 5.0
