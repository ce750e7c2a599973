"""The bench's multi-rank host logic on CPU with two gloo ranks: the timing
rule (each time is the maximum over the ranks, the whole job's throughput
counts every rank's units over that time) and the reference arm running on
rank 0 only."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    local = [10.0 + 3.0 * rank, 5.0 - rank, 7.5]
    got = bench.max_over_ranks(local, dist, "cpu")
    value = bench.job_throughput(world, 1000, 20, got[0])
    dist.barrier()
    dist.destroy_process_group()
    with open(os.path.join(out_dir, f"rank{rank}.txt"), "w") as f:
        f.write(" ".join(repr(x) for x in got + [value]))


def test_max_over_two_gloo_ranks(tmp_path):
    import torch.multiprocessing as mp
    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    rows = [list(map(float, open(tmp_path / f"rank{r}.txt").read().split())) for r in range(world)]
    for row in rows:
        assert row[:3] == [13.0, 5.0, 7.5]
        assert row[3] == pytest.approx(2 * 1000 * 20 / 13.0e-3)


def test_single_process_keeps_its_values():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks([1.5, 2.0]) == [1.5, 2.0]
    assert bench.job_throughput(1, 125000, 10, 5.0) == pytest.approx(2.5e8)


def test_reference_arm_runs_on_rank_zero_only(capsys):
    sys.path.insert(0, ROOT)
    import bench

    class Args:
        steps, warmup, gpus = 1, 0, 2
    assert bench.run_reference(Args(), 1, 2) == 0
    assert capsys.readouterr().out == ""
