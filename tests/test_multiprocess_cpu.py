"""Host logic of the multi-rank benchmark, on two gloo ranks (CPU only).

Each rank runs an independent replica (own Philox key, no collective on the
data path); the job time is the slowest rank's; the value counts the work of
every rank.  The replicas' counts come from the CPU oracle here, to show that
different ranks really draw different samples while each replica stays
reproducible.
"""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import oracle
    import qt_workloads as W
    model = W.ou2(M=2000, n=2, N=40)
    g = W.layer_grids(model)
    seed = bench.replica_seed(model, rank)
    counts = oracle.transitions(model, g, model.M, seed, oracle.PREC_F32)
    ms = 100.0 + 50.0 * rank                     # rank 1 is the slow one
    job_ms = bench.max_over_ranks(ms, dist)
    value = bench.job_value(world, model.n * model.M, job_ms)
    out[rank] = (seed, job_ms, value, counts[1].tobytes())
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_replicas_and_max_time():
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    s0, t0, v0, c0 = out[0]
    s1, t1, v1, c1 = out[1]
    assert s0 != s1                               # independent replicas
    assert t0 == t1 == 150.0                      # the slowest rank's time on every rank
    assert v0 == v1 == pytest.approx(2 * 2 * 2000 / 0.150)
    assert c0 != c1                               # different draws, different counts


def test_replica_is_reproducible():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    import oracle
    import qt_workloads as W
    model = W.ou2(M=500, n=2, N=30)
    g = W.layer_grids(model)
    a = oracle.transitions(model, g, model.M, bench.replica_seed(model, 1), oracle.PREC_F32)
    b = oracle.transitions(model, g, model.M, bench.replica_seed(model, 1), oracle.PREC_F32)
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x, y)
