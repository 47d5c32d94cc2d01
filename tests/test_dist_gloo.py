"""The benchmark's multi-rank logic on the CPU: two gloo ranks (one process each) reduce their timings the way
bench.py does under torch.distributed.run (whole-job units over the slowest rank's time; replicas only, no data
exchange)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        units = 1000.0 * (rank + 1)          # rank r integrated 1000 (r + 1) points
        ms = 10.0 + 5.0 * rank               # in 10 + 5 r ms
        bench.barrier(world)
        out[rank] = (bench.max_over_ranks(ms, world), bench.sum_over_ranks(units, world),
                     bench.whole_job_rate(units, ms, world))
    finally:
        dist.destroy_process_group()


def test_two_rank_reductions_match_the_weak_scaling_formula():
    import torch.multiprocessing as mp
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        mx, total, rate = res[r]
        assert mx == 15.0
        assert total == 3000.0
        assert abs(rate - 3000.0 / 0.015) < 1e-6
