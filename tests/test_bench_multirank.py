"""The multi-rank logic of bench.py on CPU: two gloo ranks.

bench.py runs one process per GPU under torch.distributed.run; the timed
region's length is the maximum over ranks and the units are summed (weak
scaling: every rank assembles its own replica).  Here two CPU processes
reduce through gloo exactly as the GPU ranks reduce through NCCL, and the
reference arm's non-zero ranks must exit without work or output.
"""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, elapsed, units, out_dir):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        t, u = bench.aggregate(elapsed[rank], units[rank], world, torch.device("cpu"))
        with open(os.path.join(out_dir, f"r{rank}.txt"), "w") as f:
            f.write(f"{t!r} {u!r}\n")
    finally:
        dist.destroy_process_group()


def test_aggregate_takes_max_time_and_sums_units(tmp_path):
    import torch.multiprocessing as mp
    world = 2
    elapsed = [1.25, 2.5]
    units = [1_000_000, 3_000_000]
    mp.start_processes(_rank_main, args=(world, _free_port(), elapsed, units, str(tmp_path)), nprocs=world,
                       start_method="spawn", join=True)
    for r in range(world):
        t, u = (float(x) for x in (tmp_path / f"r{r}.txt").read_text().split())
        assert t == max(elapsed)
        assert u == sum(units)


def test_single_rank_aggregate_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate(0.5, 123, 1, None) == (0.5, 123)


def test_reference_arm_other_ranks_do_nothing(capsys):
    sys.path.insert(0, ROOT)
    import argparse

    import bench
    args = argparse.Namespace(workload="n8", steps=2, warmup=1, ref_sample=1000)
    assert bench.run_reference(args, world=2, rank=1) is None
    assert capsys.readouterr().out == ""
