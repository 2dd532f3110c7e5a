"""The multi-GPU path is replicas: per-rank seeded batches, no data-path exchange, and a timing
reduction (max over ranks).  Checked here with two gloo ranks on the CPU."""
import os

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2409_07107_gb300 import replicas, scenes


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        wl = scenes.arm_cube(64, seed=replicas.rank_seed(1001, rank))
        ms = replicas.slowest_ms(10.0 + rank)
        out[rank] = (ms, replicas.job_throughput(wl.batch.B, world, ms), float(wl.batch.q.sum()))
    finally:
        dist.destroy_process_group()


def test_two_rank_replicas():
    world = 2
    port = 29500 + (os.getpid() % 1000)
    ctx = mp.get_context("spawn")
    with ctx.Manager() as man:
        out = man.dict()
        procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
        assert all(p.exitcode == 0 for p in procs)
        res = dict(out)
    assert res[0][0] == res[1][0] == 11.0                       # the slowest rank's time
    assert res[0][1] == pytest.approx(64 * 2 / 11e-3)           # all ranks' envs / slowest time
    assert res[0][2] != res[1][2]                               # each rank has its own batch


def test_single_process_fallback():
    assert replicas.slowest_ms(3.5) == 3.5
    assert replicas.rank_seed(1001, 0) == 1001 and replicas.rank_seed(1001, 1) != 1001
    assert np.isclose(replicas.job_throughput(1000, 4, 2.0), 2e6)
