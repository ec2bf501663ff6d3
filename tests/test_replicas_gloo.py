"""Multi-GPU is replicas only: each rank runs its own run, no data-path
collective; the bench takes the slowest rank's time and counts every rank's
site updates.  This checks that aggregation with two gloo ranks on CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = [100.0, 125.0][rank]
    out[rank] = bench.aggregate_over_ranks(ms, sites=1000, steps=10)
    dist.barrier()
    dist.destroy_process_group()


def test_two_replica_aggregation_uses_slowest_rank():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(2):
        ms_max, value = out[r]
        assert ms_max == 125.0
        assert value == pytest.approx(2 * 1000 * 10 / 0.125 / 1e6)


def test_single_rank_aggregation():
    import bench
    os.environ.pop("WORLD_SIZE", None)
    ms, v = bench.aggregate_over_ranks(50.0, sites=2000, steps=5)
    assert ms == 50.0 and v == pytest.approx(2000 * 5 / 0.05 / 1e6)
