"""The N > 1 path of the benchmark on CPU: two gloo ranks, each with its own
seeded shard, the max-over-ranks time and the whole-job throughput."""
import os

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, q):
    import sys
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    import bench
    from paper_1709_04145_b300 import inputs as I
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w = I.ball_chains(count=8, n_links=3, seed_base=bench.shard_seed_base(rank), n_steps=2)
    ms = 100.0 + 50.0 * rank  # rank 1 is the slow one
    ms_max = bench.max_over_ranks(ms, dist, torch.device("cpu"))
    units = w["spec"].count * w["spec"].n_links * w["n_steps"]
    value = bench.job_throughput(units, world, ms_max)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, ms_max, value, float(w["q0"].sum()), w["q0"].shape))


def test_two_gloo_ranks_shard_and_reduce():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + (os.getpid() % 1000)
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, m0, v0, s0, sh0), (r1, m1, v1, s1, sh1) = res
    assert m0 == m1 == 150.0                      # both ranks see the slowest time
    assert v0 == v1 == pytest.approx(8 * 3 * 2 * 2 / 0.150)
    assert sh0 == sh1 and s0 != s1                # same shapes, independent shards
