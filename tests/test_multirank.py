"""The N > 1 bench path on CPU: two gloo ranks, each with its own disk.

The disks shard across ranks with no data-path collective; the only
reduction is the whole-job timing (slowest rank, summed events).  Each rank
here runs a few oracle steps of its own small disk, so the per-rank work and
the aggregation are exercised without a GPU."""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import oracle
    from paper_2507_21239_gb300 import workloads as W
    P = W.benchmark_disk(dust_to_gas=0.3)
    seed = bench.rank_seed(7, rank)
    s = oracle.init_disk(P, 4 * 2 * 10, seed)
    oracle.run(P, 4, 2, s, 0.0, 50 * W.YR, 0, 3, seed)
    ms = 10.0 + rank  # stand-in per-rank time
    t, e = bench.aggregate(ms, s.events)
    out[rank] = (t, e, s.events, float(s.m.sum()))
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_by_disk():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    (t0, e0, ev0, m0), (t1, e1, ev1, m1) = out[0], out[1]
    assert t0 == t1 == 11.0                  # the slowest rank's time
    assert e0 == e1 == ev0 + ev1             # whole-job events
    assert ev0 > 0 and ev1 > 0 and m0 != m1  # independent disks
