"""Multi-rank logic of bench.py on CPU: two gloo ranks (replicas), max-over-ranks time and the
sum of rows, exactly as the GPU run combines them under torchrun."""

import os

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    def red(op):
        def f(v):
            t = torch.tensor([v], dtype=torch.float64)
            dist.all_reduce(t, op=op)
            return float(t.item())
        return f

    ms_local = 100.0 + 50.0 * rank  # rank 1 is the slow one
    rows_local = 1000 * (rank + 1)
    ms, value = bench.aggregate(ms_local, rows_local, 4, red(dist.ReduceOp.MAX), red(dist.ReduceOp.SUM))
    out[rank] = (ms, value)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_aggregate():
    port = 29500 + (os.getpid() % 1000)
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    for r in (0, 1):
        ms, value = res[r]
        assert ms == pytest.approx(150.0)
        assert value == pytest.approx((1000 + 2000) * 4 / 0.150)


def test_single_rank_aggregate():
    import bench

    ms, value = bench.aggregate(20.0, 500, 10)
    assert ms == 20.0 and value == pytest.approx(500 * 10 / 0.020)
