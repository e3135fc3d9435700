"""The replica path of bench.py with two gloo ranks on the CPU: every rank
reports the slowest rank's times and the whole-job throughput."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
dist = pytest.importorskip("torch.distributed")
mp = pytest.importorskip("torch.multiprocessing")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        dist.barrier()
        t_dev, wall, value = bench.combine_ranks(1.0 + rank, 2.0 + 0.5 * rank, 3, world, dist)
        dist.barrier()
        with open(os.path.join(out, f"rank{rank}.txt"), "w") as f:
            f.write(f"{t_dev} {wall} {value}")
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_slowest_rank_and_throughput(tmp_path):
    world = 2
    mp.spawn(_rank, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    for r in range(world):
        t_dev, wall, value = map(float, (tmp_path / f"rank{r}.txt").read_text().split())
        assert t_dev == 2.0 and wall == 2.5
        assert value == pytest.approx(3 * world / 2.0)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.combine_ranks(0.5, 0.7, 4, 1) == (0.5, 0.7, 8.0)
