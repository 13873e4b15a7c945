"""Multi-process replica path of bench.py on CPU ranks (gloo, world size 2).

The solver does not shard across GPUs: with N GPUs each rank solves its own
replica and the job time is the slowest rank's.  This checks that aggregation
and that the replicas of one seeded problem agree (the oracle stands in for
the per-rank solver on CPU ranks).
"""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from oracle import rks as R
    from paper_2508_05400_gb300 import inputs as I
    A = I.convdiff_2d(20, 20, 1.0, 20.0, 10.0)
    res = R.rks(A.to_scipy(), 4, 12, 40, I.start_vector(A.n, 1), zeta=8, seed=0, which="LR",
                tol=1e-12)
    per_rank_ms = [100.0 + 50.0 * rank, 7.0 * (rank + 1)]
    agg = bench.reduce_max_over_ranks(per_rank_ms, "cpu", dist, world)
    lam = torch.tensor(np.stack([res.eigvals.real, res.eigvals.imag]))
    gathered = [torch.zeros_like(lam) for _ in range(world)]
    dist.all_gather(gathered, lam)
    out[rank] = (agg, [g.numpy() for g in gathered])
    dist.destroy_process_group()


def test_replicas_two_gloo_ranks():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(240)
        assert p.exitcode == 0
    for r in range(world):
        agg, lams = out[r]
        assert agg == [150.0, 14.0]            # slowest rank bounds each figure
        assert np.array_equal(lams[0], lams[1])  # replicas of one seeded problem agree
