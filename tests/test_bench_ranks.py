"""Host side of the multi-GPU bench: N independent replicas, no data-path
collective.  Two gloo ranks on the CPU check the job-level aggregation that
`bench.py` runs under torchrun (slowest rank's time, units of all ranks) and
that every rank draws its own problems."""
import multiprocessing as mp
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r pretends to have taken 10+r ms for the device steps and
        # 3-r s for the host steps: the job takes the slowest of each.
        ms, e2e_s = bench.max_over_ranks(dist, [10.0 + rank, 3.0 - rank])
        sets = bench.workload(4096, rank)
        pts = sum(len(p) for p in sets)
        value = bench.job_mpts(pts, world, 5, ms / 1e3)
        digest = [int(np.asarray(p, dtype=np.int64).sum()) for p in sets]
        q.put((rank, ms, e2e_s, pts, value, digest))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_like_the_bench():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = {}
    for _ in range(world):
        r = q.get(timeout=120)
        res[r[0]] = r
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in range(world):
        _, ms, e2e_s, pts, value, _ = res[r]
        assert ms == 11.0            # the slower rank's device time
        assert e2e_s == 3.0          # the slower rank's host time
        assert pts == 2 * 4096
        # every rank's points over the slowest rank's time
        assert value == pytest.approx(world * pts * 5 / 0.011 / 1e6)
    # independent problems on each rank
    assert res[0][5] != res[1][5]


def test_single_process_aggregation_is_identity():
    import bench
    assert bench.max_over_ranks(None, [1.5, 2]) == [1.5, 2.0]
    assert bench.job_mpts(40_000_000, 1, 20, 0.04) == pytest.approx(20_000.0)
    a0 = bench.workload(1000, 0)
    assert [len(p) for p in a0] == [1000, 1000]
