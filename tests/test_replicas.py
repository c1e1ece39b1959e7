"""The multi-GPU path of bench.py is independent replicas (no data-path collective): the
reported value is every rank's units over the slowest rank's time.  Two gloo ranks on the
CPU check the max-over-ranks aggregation."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, totals, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        value, slowest = bench.aggregate_replicas(totals[rank], 1000, world,
                                                  lambda x: bench.max_over_ranks(torch, dist, x, torch.device("cpu")))
        out[rank] = (value, slowest)
    finally:
        dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_two_replicas_report_units_over_the_slowest_rank():
    world, totals = 2, [10.0, 14.0]                     # ms of the timed region on each rank
    out = mp.get_context("spawn").Manager().dict()
    mp.start_processes(_rank, args=(world, _free_port(), totals, out), nprocs=world, start_method="spawn")
    for r in range(world):
        value, slowest = out[r]
        assert slowest == 14.0
        assert abs(value - world * 1000 / 14e-3) < 1e-6


def test_single_rank_needs_no_collective():
    value, slowest = bench.aggregate_replicas(8.0, 400, 1, lambda x: x)
    assert slowest == 8.0 and abs(value - 400 / 8e-3) < 1e-9
