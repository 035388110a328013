"""The N > 1 path of the benchmark on CPU: every rank is a replica that times
its own work; the job's time is the slowest rank's (all_reduce MAX over
gloo, world size 2) and its throughput the units of all ranks over it."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out_dir):
    import torch.distributed as tdist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    tdist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        my_ms = [12.5, 20.0][rank]
        ms = bench.max_over_ranks(my_ms, world, device="cpu")
        rate = bench.job_rate(1000.0, world, ms)
        with open(os.path.join(out_dir, f"r{rank}"), "w") as f:
            f.write(f"{ms} {rate}")
        tdist.barrier()
    finally:
        tdist.destroy_process_group()


def test_two_replicas_report_the_slowest_rank(tmp_path):
    mp = pytest.importorskip("torch.multiprocessing")
    world = 2
    mp.start_processes(_rank, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    for r in range(world):
        ms, rate = map(float, (tmp_path / f"r{r}").read_text().split())
        assert ms == 20.0
        assert rate == pytest.approx(world * 1000.0 / 0.020)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.0, 1) == 3.0
    assert bench.job_rate(10.0, 1, 2.0) == pytest.approx(5000.0)
