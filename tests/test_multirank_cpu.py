"""Multi-rank host logic on CPU (gloo, world size 2): the benchmark's
replicas-only scaling takes the max of the per-rank times and sums the trials
of all ranks, with no collective on the data path.  The aggregation is the
same code bench.py runs under torchrun."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = 100.0 + 50.0 * rank  # per-rank timed region
    agg = bench.aggregate_ranks(ms, sites=1000, steps=4, dist_mod=dist, device="cpu")
    out[rank] = agg
    dist.destroy_process_group()


def test_weak_scaling_aggregation_two_ranks():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(60)
            assert p.exitcode == 0
        for r in range(world):
            ms_max, value = out[r]
            assert ms_max == pytest.approx(150.0)
            assert value == pytest.approx(1000 * 4 * world / 0.150)
