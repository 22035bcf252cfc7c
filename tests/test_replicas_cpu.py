"""Multi-rank host logic of bench.py on CPU: two gloo ranks, each running
its own replica, agree on the slowest rank's time and on the whole-job
rate; the reference arm runs on rank 0 only."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = 10.0 * (rank + 1)                     # rank 1 is the slower replica
    got = bench.reduce_max(local_ms)
    rate = bench.job_rate(1000.0, world, got)
    ref = bench.run_reference(type("A", (), {"workload": "pr1", "points": 0, "steps": 1, "warmup": 0})(),
                              rank, world) if rank == 1 else "skipped"
    out[rank] = (got, rate, ref)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_max_time_and_rate():
    world = 2
    out = mp.get_context("spawn").Manager().dict()
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    for rank in range(world):
        got, rate, _ = out[rank]
        assert got == 20.0
        assert rate == pytest.approx(2 * 1000.0 / 0.020)
    assert out[1][2] is None                         # the reference arm is rank 0's job


def test_single_process_reduce_is_identity():
    import bench
    assert bench.reduce_max(3.5) == 3.5
    assert bench.job_rate(10.0, 1, 1000.0) == 10.0


def test_clock_sample_summary():
    """The clocks record beside a bench number: median SM clock under load,
    maximum clock, and only the throttle reasons reported Active."""
    import bench
    rows = "\n".join([
        "345, 2032, 120.5, Not Active, Not Active, Not Active, Not Active",      # idle before the region
        "2032, 2032, 900.1, Not Active, Not Active, Not Active, Not Active",
        "2017, 2032, 1099.0, Not Active, Not Active, Not Active, Active",         # power cap: kept, noted
        "2032, 2032, 950.0, Not Active, Not Active, Not Active, Not Active",
        "[N/A], 2032, 10.0, Not Active, Not Active, Not Active, Not Active",      # unreadable sample skipped
    ])
    s = bench.summarize_clock_samples(rows)
    assert s == {"sm_mhz": 2032.0, "sm_max_mhz": 2032.0, "samples": 4, "reasons": ["sw_power_cap"]}
    hot = bench.summarize_clock_samples("1500, 2032, 1000, Active, Not Active, Active, Not Active")
    assert hot["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]
    assert bench.summarize_clock_samples("") is None
