"""Host logic of the N-replica benchmark, run as two gloo ranks on the CPU.

Each rank of an N-GPU run processes the whole workload (the units are independent problems, so
there is no data-path collective).  The timing is the slowest rank's, and the reported throughput
counts every rank's evaluations.  The reference arm runs on rank 0 alone; the other ranks return
without work.
"""
import argparse
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def rank_main(rank, world, port, times):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        dist.barrier()
        slowest = bench.max_over_ranks(times[rank], torch.device("cpu"), world)
        assert slowest == max(times), (rank, slowest)
        assert bench.replica_throughput(world, 5, slowest) == pytest.approx(world * 5 / max(times))
        if rank != 0:
            args = argparse.Namespace(workload="tiny32", steps=1, warmup=0, gpus=world)
            assert bench.run_reference(args, rank) is None
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_rank_max_over_ranks_and_replica_throughput():
    import torch.multiprocessing as mp

    times = [1.25, 2.5]
    mp.start_processes(rank_main, args=(2, free_port(), times), nprocs=2, join=True, start_method="spawn")


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks(0.75, torch.device("cpu"), 1) == 0.75
    assert bench.replica_throughput(1, 5, 2.0) == 2.5
