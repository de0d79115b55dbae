"""Parity of every pipeline stage, called through the C ABI, against the CPU
oracle on the same seeded inputs.  Integer/index work: bit-exact."""
import numpy as np
import pytest

import oracle
from paper_1508_05931_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ctx(hull_lib):
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    c = hull_lib.Context(0, collect_stats=True)
    yield c
    c.close()


def dev(a):
    if not isinstance(a, np.ndarray):
        a = np.asarray(a, dtype=np.int32).reshape(-1, 2)
    return torch.as_tensor(np.ascontiguousarray(a)).cuda()


def rand_pts(rng, n, span):
    return rng.integers(-span, span + 1, size=(n, 2)).astype(np.int32)


SIZES = [1, 2, 3, 7, 31, 4095, 4096, 4097, 8191, 12289, 65537, 300001]


@pytest.mark.parametrize("n", SIZES)
@pytest.mark.parametrize("span", [0, 2, 1000, 1 << 29])
def test_extremes_parity(ctx, n, span):
    rng = np.random.default_rng(n * 31 + span % 1009)
    pts = rand_pts(rng, n, span)
    assert ctx.stage_extremes(dev(pts)).tolist() == oracle.extremes(pts).tolist()


def test_extremes_unaligned_view(ctx):
    rng = np.random.default_rng(5)
    pts = rand_pts(rng, 100001, 50)
    t = dev(pts)
    view = t[1:]                       # 8-byte but not 16-byte aligned
    assert view.data_ptr() % 16 == 8
    assert ctx.stage_extremes(view).tolist() == oracle.extremes(pts[1:]).tolist()


@pytest.mark.parametrize("n", SIZES)
@pytest.mark.parametrize("gen", ["square", "disk", "ties", "grid"])
def test_filter_parity(ctx, n, gen):
    rng = np.random.default_rng(n + 17)
    if gen == "square":
        pts = W.uniform_square(n, 1 << 29, n)
    elif gen == "disk":
        pts = W.uniform_disk(n, 1e6, n)
    elif gen == "ties":
        pts = rand_pts(rng, n, 3)
    else:
        k = max(1, int(np.sqrt(n)))
        pts = W.filled_grid(k, k)[:n]
    keep = ctx.stage_filter(dev(pts)).cpu().numpy()
    assert np.array_equal(keep, oracle.quad_filter(pts))


def test_filter_unaligned_view(ctx):
    pts = W.uniform_disk(50001, 1e7, 3)
    view = dev(pts)[1:]
    assert view.data_ptr() % 16 == 8
    keep = ctx.stage_filter(view).cpu().numpy()
    assert np.array_equal(keep, oracle.quad_filter(pts[1:]))


@pytest.mark.parametrize("m", [1, 2, 100, 4095, 4096, 4097, 100003, 1000001])
@pytest.mark.parametrize("kind", ["random", "equal", "sorted", "reverse", "lowbits"])
def test_sort_parity(ctx, m, kind):
    rng = np.random.default_rng(m)
    if kind == "random":
        keys = rng.integers(0, 2 ** 63, size=m, dtype=np.uint64) * np.uint64(2) + rng.integers(0, 2, size=m).astype(np.uint64)
    elif kind == "equal":
        keys = np.full(m, 12345, dtype=np.uint64)
    elif kind == "sorted":
        keys = np.sort(rng.integers(0, 2 ** 40, size=m).astype(np.uint64))
    elif kind == "reverse":
        keys = np.sort(rng.integers(0, 2 ** 40, size=m).astype(np.uint64))[::-1].copy()
    else:
        keys = rng.integers(0, 16, size=m).astype(np.uint64)
    vals = rng.permutation(m).astype(np.int32)
    kt = dev(keys.view(np.int64))
    vt = dev(vals)
    ctx.stage_sort(kt, vt)
    order = np.argsort(keys, kind="stable")
    assert np.array_equal(kt.cpu().numpy().view(np.uint64), keys[order])
    assert np.array_equal(vt.cpu().numpy(), vals[order])


def _bucket_keys(rng, m, kind):
    if kind == "random":            # full 64-bit keys: many small bins, insertion path
        return rng.integers(0, 2 ** 63, size=m, dtype=np.uint64) * np.uint64(2) + rng.integers(0, 2, size=m).astype(np.uint64)
    if kind == "equal":             # one bin: bitonic path up to the group cap, then the radix passes
        return np.full(m, 12345, dtype=np.uint64)
    if kind == "lowbits":           # 16 distinct keys: crowded sub-bins
        return rng.integers(0, 16, size=m).astype(np.uint64)
    if kind == "dups":              # ~1000 distinct keys, each a bin of its own
        return (rng.integers(0, 1000, size=m).astype(np.uint64) << np.uint64(40)) + np.uint64(7)
    if kind == "bigbin":            # a third of the keys in the first bin: split once more
        k = rng.integers(0, 2 ** 61, size=m, dtype=np.uint64)
        third = m // 3
        k[:third] = rng.integers(0, 2 ** 47, size=third, dtype=np.uint64)
        return rng.permutation(k)
    if kind == "lattice":           # the pipeline's keys of a small uniform square
        pts = W.uniform_square(m, 1 << 20, m)
        x = pts[:, 0].astype(np.int64) - pts[:, 0].min()
        y = pts[:, 1].astype(np.int64) - pts[:, 1].min()
        yb = int(y.max()).bit_length()
        return ((x << yb) | y).astype(np.uint64)
    raise ValueError(kind)


@pytest.mark.parametrize("m", [1, 2, 100, 4097, 8192, 8193, 100003, 1000001])
@pytest.mark.parametrize("kind", ["random", "equal", "lowbits", "dups", "bigbin", "lattice"])
def test_bucket_sort_parity(ctx, hull_lib, m, kind):
    """The pipeline's bucket sort orders (key, value) pairs by key, then
    value; with values ascending in input order (as the first round's
    survivor indices are) that is the stable sort by key."""
    rng = np.random.default_rng(m * 13 + len(kind))
    keys = _bucket_keys(rng, m, kind)
    vals = np.arange(m, dtype=np.int32)
    kt = dev(keys.view(np.int64))
    vt = dev(vals)
    fell_back = ctx.stage_bucket_sort(kt, vt)
    order = np.argsort(keys, kind="stable")
    assert np.array_equal(kt.cpu().numpy().view(np.uint64), keys[order])
    assert np.array_equal(vt.cpu().numpy(), vals[order])
    # Only a bin of more keys than one block sorts in shared memory that its
    # next key bits cannot split (equal keys here) hands the pairs to the
    # radix passes.
    cap = hull_lib.hull_bucket_group_cap()
    expect_fb = (kind == "equal" and m > cap) or (kind == "lowbits" and m > 16 * cap)
    assert fell_back == expect_fb


def test_bucket_sort_values_break_ties(ctx):
    """Among equal keys the smaller value comes first, whatever the input order."""
    rng = np.random.default_rng(3)
    m = 50000
    keys = rng.integers(0, 300, size=m).astype(np.uint64) << np.uint64(33)
    vals = rng.permutation(m).astype(np.int32)
    kt, vt = dev(keys.view(np.int64)), dev(vals)
    assert not ctx.stage_bucket_sort(kt, vt)
    order = np.lexsort((vals, keys))
    assert np.array_equal(kt.cpu().numpy().view(np.uint64), keys[order])
    assert np.array_equal(vt.cpu().numpy(), vals[order])


def _sorted_input(pts):
    srt = oracle.sort_survivors(pts, np.arange(len(pts)))
    return pts[srt], srt


@pytest.mark.parametrize("n", [2, 3, 5, 64, 4096, 4097, 20000, 300001])
@pytest.mark.parametrize("span", [1, 3, 100, 1 << 29])
def test_second_round_parity(ctx, n, span):
    rng = np.random.default_rng(n * 7 + span % 101)
    pts = rand_pts(rng, n, span)
    xy, srt = _sorted_input(pts)
    lo_ref, up_ref, _ = oracle.second_round(pts, srt)
    lo, up = ctx.stage_second_round(xy, srt)
    assert np.array_equal(lo.cpu().numpy(), lo_ref)
    assert np.array_equal(up.cpu().numpy(), up_ref)


@pytest.mark.parametrize("n", [1, 2, 4097, 65537, 1_000_003])
@pytest.mark.parametrize("gen", ["square", "disk", "ties"])
def test_sorted_survivors_parity(ctx, n, gen):
    """Steps 1-4 on the device (extremes, quad filter, stable compaction,
    radix sort): the survivors in (x, y, index) order, bit-exact."""
    rng = np.random.default_rng(n + 5)
    pts = {"square": lambda: W.uniform_square(n, 1 << 29, n), "disk": lambda: W.uniform_disk(n, 2.0 ** 29, n),
           "ties": lambda: rand_pts(rng, n, 5)}[gen]()
    ref = oracle.sort_survivors(pts, oracle.quad_filter(pts))
    xy, idx = ctx.stage_sorted_survivors(dev(pts))
    assert np.array_equal(idx.cpu().numpy(), ref)
    assert np.array_equal(xy.cpu().numpy(), pts[ref])


@pytest.mark.parametrize("n", [2, 5, 4097, 300001])
@pytest.mark.parametrize("span", [1, 100, 1 << 29])
@pytest.mark.parametrize("bs", [1, 7, 1024])
def test_second_round_chunked_parity(ctx, n, span, bs):
    """Section 3.4's chunked second round on the device (one thread per run,
    one block per region) equals the oracle's, list for list."""
    rng = np.random.default_rng(n * 3 + span % 97 + bs)
    pts = rand_pts(rng, n, span)
    xy, srt = _sorted_input(pts)
    lo_ref, up_ref, _ = oracle.second_round_chunked(pts, srt, bs)
    lo, up = ctx.stage_second_round_chunked(xy, srt, bs)
    assert np.array_equal(lo.cpu().numpy(), lo_ref)
    assert np.array_equal(up.cpu().numpy(), up_ref)


def test_second_round_chunked_golden_and_paper_shapes(ctx):
    import json
    import os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "second_round_chunked_trace.json")))
    names, P, perm = g["names"], g["points"], g["index_permutation"]
    pts = np.zeros((len(P), 2), np.int32)
    for k, j in enumerate(perm):
        pts[j] = P[k]
    name_of = {perm[k]: names[k] for k in range(len(names))}
    xy, srt = _sorted_input(pts)
    lo, up = ctx.stage_second_round_chunked(xy, srt, g["block_size"])
    assert [name_of[int(i)] for i in lo.cpu().numpy()] == g["expected_lower_kept"]
    assert [name_of[int(i)] for i in up.cpu().numpy()] == g["expected_upper_kept"]
    for pts in (W.uniform_square(1_000_000, 1 << 29, 61), W.uniform_disk(1_000_000, 2.0 ** 29, 62)):
        srt = oracle.sort_survivors(pts, oracle.quad_filter(pts))
        lo_ref, up_ref, _ = oracle.second_round_chunked(pts, srt, 1024)
        lo, up = ctx.stage_second_round_chunked(pts[srt], srt, 1024)
        assert np.array_equal(lo.cpu().numpy(), lo_ref) and np.array_equal(up.cpu().numpy(), up_ref)


def test_second_round_golden_trace(ctx):
    import json
    import os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "second_round_trace.json")))
    names, P, perm = g["names"], g["points"], g["index_permutation"]
    pts = np.zeros((len(P), 2), np.int32)
    for k, j in enumerate(perm):
        pts[j] = P[k]
    name_of = {perm[k]: names[k] for k in range(len(names))}
    xy, srt = _sorted_input(pts)
    lo, up = ctx.stage_second_round(xy, srt)
    assert [name_of[int(i)] for i in lo.cpu().numpy()] == g["expected_lower_kept"]
    assert [name_of[int(i)] for i in up.cpu().numpy()] == g["expected_upper_kept"]
    h = ctx.compute(dev(pts)).cpu().numpy()
    assert [name_of[int(i)] for i in h] == g["expected_hull_ccw"]


@pytest.mark.parametrize("m", [2, 3, 9, 33, 4095, 4096, 4097, 8193, 20000, 70001])
@pytest.mark.parametrize("gen", ["random", "convex", "ties"])
def test_chain_parity(ctx, m, gen):
    rng = np.random.default_rng(m + 3)
    if gen == "random":
        u = np.unique(rand_pts(rng, m * 2, 1 << 29), axis=0)[:m]
    elif gen == "convex":
        t = np.sort(rng.choice(np.arange(-(1 << 16), 1 << 16), size=m, replace=False)).astype(np.int64)
        u = np.stack([t, t * t // 8 - (1 << 28)], axis=1).astype(np.int32)
    else:
        u = np.unique(rand_pts(rng, m * 4, 40), axis=0)[:m]
    if len(u) < 2:
        pytest.skip("degenerate draw")
    u = np.ascontiguousarray(u.astype(np.int32))
    lo, up = ctx.stage_chain(u)
    assert np.array_equal(lo, oracle.chain(u, +1))
    assert np.array_equal(up, oracle.chain(u, -1))
