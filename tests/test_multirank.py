"""Host logic of the multi-GPU path (replicas: every rank filters its own copy of the
batch, no data-path collective) on world_size-2 gloo process groups on the CPU: the
timing reduction takes the slowest rank, the whole-job rate counts every rank's
samples, and the reference arm runs on rank 0 only."""
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, loc = bench.dist_env()
        assert (w, r, loc) == (world, rank, rank)
        mine = 1.5 + rank               # this rank's step time (ms)
        slowest = bench.max_over_ranks(mine, world, device="cpu")
        rate = bench.whole_job_rate(1000, world, slowest)
        # the reference arm prints on rank 0 only: other ranks return without work
        called = []
        if rank != 0:
            class A:
                workload = "allpole2_4x4096"
            import oracle
            real = oracle.forward
            oracle.forward = lambda *a, **k: called.append(1)
            try:
                bench.run_reference(A(), world, rank)
            finally:
                oracle.forward = real
        out[rank] = (slowest, rate, len(called))
    finally:
        dist.destroy_process_group()


def test_replica_timing_two_ranks():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    mp.start_processes(_rank_main, args=(world, port, out), nprocs=world, join=True,
                       start_method="spawn")
    for r in range(world):
        slowest, rate, called = out[r]
        assert slowest == pytest.approx(2.5)                  # max over ranks
        assert rate == pytest.approx(1000 * 2 / 2.5e-3 / 1e9)  # both ranks' samples
        assert called == 0
