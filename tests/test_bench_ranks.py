"""The whole-job figures of bench.py under torchrun: the slowest rank's time and
the RHS solved on all ranks together, over a world-size-2 gloo process group on
the CPU (no GPU)."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        ms, solved = bench.reduce_over_ranks(10.0 + 5.0 * rank, 128 - rank, world)
        out[rank] = (ms, solved)
    finally:
        dist.destroy_process_group()


def test_slowest_rank_and_total_solved_over_two_ranks():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        mp.start_processes(_rank, args=(2, _free_port(), out), nprocs=2, join=True, start_method="spawn")
        res = dict(out)
    assert res[0] == res[1] == (15.0, 255)


def test_single_rank_is_unchanged():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_over_ranks(7.5, 42, 1) == (7.5, 42)


def test_roofline_fields_from_a_profile():
    """roofline_of: algorithmic bytes per launch over the average launch time against
    the measured HBM peak; the tensor companion against the sustained BF16 peak; DRAM
    traffic per launch from the committed ncu summary of the class."""
    sys.path.insert(0, ROOT)
    import bench
    hbm, bf16_s, src = bench.peaks(sustained=True)
    prof = {"conv3x3_tc": (2000.0, 1000, 5.0e12), "cnn_io": (100.0, 10, 0.0)}
    flops = {"conv3x3_tc": 7.0e14}
    r = bench.roofline_of(prof, flops)
    assert r["kernel"] == "conv3x3_tc" and r["bound"] == "hbm"
    assert abs(r["achieved"] - 5.0e12 / 2.0 / 1e9) < 1e-6          # GB/s over 2 s
    assert abs(r["frac"] - r["achieved"] / hbm) < 1e-12
    assert abs(r["tensor"]["achieved"] - 7.0e14 / 2.0 / 1e12) < 1e-9
    assert abs(r["tensor"]["frac"] - r["tensor"]["achieved"] / bf16_s) < 1e-12
    assert r["traffic"] == bench.traffic_from_profiles("conv3x3_tc") and r["traffic"] > 0
    assert abs(r["algorithmic_bytes_per_launch"] - 5.0e9) < 1e-3
