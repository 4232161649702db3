"""The multi-process path of the benchmark, on CPU with two gloo ranks.

bench.py --gpus N runs N independent replicas (one problem per rank, seeded by
rank; no data-path collective): each rank times its own steps, the job's time is
the slowest rank's, and the whole-job value counts the units of all ranks. Only
rank 0 runs the reference arm. These are the parts that do not need a GPU.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank: int, world: int, port: int) -> None:
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port),
                       "RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    import bench
    import synth

    w, r, local = bench.dist_env()
    assert (w, r, local) == (world, rank, rank)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # the slowest rank's time is every rank's result
        ms = bench.max_over_ranks(10.0 + 5.0 * rank, world, "cpu")
        assert ms == 10.0 + 5.0 * (world - 1)
        assert bench.whole_job_value(100.0, world, ms) == pytest.approx(100.0 * world / (ms / 1e3))
        # replicas: every rank solves its own problem (seeded by rank)
        p = synth.large_problem(seed=rank, n=256, iters=1)
        mine = torch.tensor([float(np.asarray(p.X, np.float64).sum())])
        every = [torch.zeros(1) for _ in range(world)]
        dist.all_gather(every, mine)
        assert len({float(t.item()) for t in every}) == world
        # the reference arm runs on rank 0 only; the others return without work
        if rank != 0:

            class Args:
                steps, warmup, gpus = 1, 0, world

            assert bench.run_reference(Args()) == 0
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_time_and_aggregate_like_the_benchmark():
    world = 2
    mp.spawn(_rank_main, args=(world, _free_port()), nprocs=world, join=True)


def test_single_process_needs_no_collective():
    import bench
    assert bench.max_over_ranks(12.5, 1, "cpu") == 12.5
    assert bench.whole_job_value(3e9, 1, 1000.0) == pytest.approx(3e9)
