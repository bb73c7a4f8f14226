"""The multi-rank path on CPU: two gloo ranks, each with its own shard of the
counter-based event stream, combine their event sums with the benchmark's
reductions; the result equals the event sum of the whole range.

Events are independent (Sec. 3: every event's |M|^2 is computed on its own),
so the only exchange is the final sum of (sum w me, sum (w me)^2, N) and the
job time is the slowest rank's.  The per-rank work here is the oracle (CPU).
"""
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

WORLD = 2
NEVT = 48  # events per rank
PROC, ECM = 1, 500.0


def free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def shard_sums(rank: int):
    import bench
    import oracle
    from paper_2106_12631_gb300 import inputs as I
    seed = I.seed_of("ee_mumu")
    rnd = I.uniforms(seed, 8, NEVT, first_event=bench.shard_first_event(rank, NEVT))
    mom, wgt = oracle.rambo(PROC, rnd, ECM)
    me = oracle.me(PROC, mom)
    return rnd, oracle.event_sum(me, wgt)


def worker(rank: int, port: int, out):
    import bench
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=WORLD)
    try:
        rnd, s = shard_sums(rank)
        sums = torch.tensor(s, dtype=torch.float64)
        bench.sum_over_ranks(sums, WORLD)
        t = bench.max_over_ranks(0.25 + rank, WORLD, torch.device("cpu"))
        out[rank] = (sums.numpy().copy(), t, rnd[:, 0].copy())
    finally:
        dist.destroy_process_group()


@pytest.fixture(scope="module")
def results():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    mp.start_processes(worker, args=(free_port(), out), nprocs=WORLD, join=True, start_method="spawn")
    return dict(out)


def test_ranks_agree_and_match_whole_range(results):
    import oracle
    from paper_2106_12631_gb300 import inputs as I
    (s0, t0, _), (s1, t1, _) = results[0], results[1]
    np.testing.assert_array_equal(s0, s1)
    assert t0 == t1 == 1.25  # the slowest rank's time
    rnd = I.uniforms(I.seed_of("ee_mumu"), 8, WORLD * NEVT)
    mom, wgt = oracle.rambo(PROC, rnd, ECM)
    whole = oracle.event_sum(oracle.me(PROC, mom), wgt)
    assert s0[2] == WORLD * NEVT
    np.testing.assert_allclose(s0[:2], whole[:2], rtol=1e-14, atol=0)


def test_shards_are_disjoint_ranges(results):
    from paper_2106_12631_gb300 import inputs as I
    whole = I.uniforms(I.seed_of("ee_mumu"), 8, WORLD * NEVT)
    for r in range(WORLD):
        np.testing.assert_array_equal(results[r][2], whole[:, r * NEVT])
