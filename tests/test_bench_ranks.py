"""bench.py with --gpus N > 1 runs N independent replicas; its whole-job
figures are the slowest rank's time and the sum of the ranks' flops.  The
aggregation runs here on two CPU ranks over gloo."""
import os

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _rank(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        ms = [120.0, 150.0, 90.0][rank]
        flops = [1.0e12, 2.0e12, 4.0e12][rank]
        out[rank] = bench.aggregate_ranks(ms, flops, world, device="cpu")
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_replica_aggregation_on_cpu_ranks(world):
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
        assert all(p.exitcode == 0 for p in procs)
        res = dict(out)
    ms_max = max([120.0, 150.0, 90.0][:world])
    flops_all = sum([1.0e12, 2.0e12, 4.0e12][:world])
    assert all(res[r] == (ms_max, flops_all) for r in range(world))


def test_single_rank_is_its_own_figures():
    import bench
    assert bench.aggregate_ranks(12.5, 3.0e9, 1) == (12.5, 3.0e9)
