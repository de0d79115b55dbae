"""One hull sharded across ranks (paper_1508_05931_gb300/shard.py): two gloo
ranks on the CPU each take a contiguous shard, gather their hulls'
vertices and merge them; every rank's result must equal the oracle's hull
of the whole input, bit-exact, including duplicate points held by both
shards (smallest global index), a shard with no points, collinear inputs
and shards whose hulls are nested.  The ranks' hull routine is the oracle
(test infrastructure, injected), so this checks the gather and the merge;
the CUDA pipeline's part is checked in one process on the GPU."""
import multiprocessing as mp
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1508_05931_gb300 import shard  # noqa: E402
from paper_1508_05931_gb300 import workloads as W  # noqa: E402


def cases():
    rng = np.random.default_rng(5)
    few = rng.integers(-50, 51, size=(30, 2)).astype(np.int32)
    dup = few[rng.integers(0, 30, size=4000)]                  # duplicates across the shards
    nested = np.concatenate([W.uniform_disk(3000, 1e3, 6), W.uniform_disk(3000, 1e6, 7)])
    t = np.arange(-400, 400)
    return {
        "square": W.uniform_square(20000, 1 << 29, 1),
        "disk": W.uniform_disk(20000, 2.0 ** 29, 2),
        "circle": W.near_circle(5000, 2.0 ** 16, 3),
        "dup": dup,
        "nested": nested,                                   # rank 0's hull lies inside rank 1's
        "collinear": np.stack([t * 3, t * 5], axis=1).astype(np.int32),
        "identical": np.full((500, 2), 9, np.int32),
        "one": np.array([[4, 4]], np.int32),               # rank 0 holds nothing
        "lattice": W.parabola_lattice(700),
    }


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        out = {}
        for name, pts in cases().items():
            lo, hi = shard.shard_bounds(len(pts), rank, world)
            out[name] = shard.sharded_hull(pts[lo:hi], lo, hull_fn=oracle.hull).tolist()
        q.put((rank, out))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_merge_equals_oracle_hull_of_union():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = {}
    for _ in range(world):
        r, out = q.get(timeout=180)
        res[r] = out
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for name, pts in cases().items():
        ref = oracle.hull(pts).tolist()
        assert res[0][name] == ref, name
        assert res[1][name] == ref, name


def test_merge_of_many_shards_without_a_process_group():
    """The merge alone over 1..7 contiguous shards, every split point."""
    for name, pts in cases().items():
        ref = oracle.hull(pts).tolist()
        for world in (1, 2, 3, 7):
            parts = []
            for r in range(world):
                lo, hi = shard.shard_bounds(len(pts), r, world)
                parts.append(shard.local_vertices(pts[lo:hi], lo, oracle.hull))
            assert shard.merge(parts, oracle.hull).tolist() == ref, (name, world)


def test_merge_keeps_the_smallest_index_of_a_shared_point():
    pts = np.array([[0, 0], [5, 0], [0, 5], [0, 0], [5, 0], [0, 5], [1, 1]], np.int32)
    parts = [shard.local_vertices(pts[:3], 0, oracle.hull), shard.local_vertices(pts[3:], 3, oracle.hull)]
    assert shard.merge(parts, oracle.hull).tolist() == [0, 1, 2] == oracle.hull(pts).tolist()


def test_shard_bounds_cover_the_input():
    for n in (0, 1, 7, 1000):
        for world in (1, 2, 3, 8):
            b = [shard.shard_bounds(n, r, world) for r in range(world)]
            assert b[0][0] == 0 and b[-1][1] == n
            assert all(b[i][1] == b[i + 1][0] for i in range(world - 1))


@pytest.mark.gpu
def test_merge_through_the_cuda_pipeline(hull_lib):
    """Shards of the 20M square and disk, each shard's hull and the merge by
    the CUDA pipeline in one process: the oracle's hull of the whole set."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    with hull_lib.Context(0) as ctx:
        fn = shard._default_hull(ctx)
        for pts in (W.paper_square(), W.paper_disk(), cases()["dup"], cases()["nested"]):
            ref = oracle.hull(pts).tolist()
            for world in (2, 4):
                parts = []
                for r in range(world):
                    lo, hi = shard.shard_bounds(len(pts), r, world)
                    parts.append(shard.local_vertices(pts[lo:hi], lo, fn))
                assert shard.merge(parts, fn).tolist() == ref
