"""Batched mode: every instance's hull equals the oracle's, bit-exact, in a
single hull_compute_batched call (mixed sizes across both size buckets,
empty and degenerate instances, the uneven-size batch generator)."""
import os

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
    c = hull_lib.Context(0)
    yield c
    c.close()


def run_batch(ctx, parts, cap=None):
    offs = np.zeros(len(parts) + 1, np.int64)
    offs[1:] = np.cumsum([len(p) for p in parts])
    pts = np.concatenate(parts, axis=0) if parts else np.zeros((0, 2), np.int32)
    t = torch.as_tensor(np.ascontiguousarray(pts, dtype=np.int32)).cuda()
    out = torch.empty(max(cap if cap is not None else len(pts), 1), dtype=torch.int32, device="cuda")
    o, oo = ctx.compute_batched(t, torch.as_tensor(offs), out=out)
    return o.cpu().numpy(), oo.cpu().numpy()


def check(parts, o, oo):
    assert len(oo) == len(parts) + 1 and oo[0] == 0
    for i, p in enumerate(parts):
        got = o[oo[i]:oo[i + 1]]
        assert got.tolist() == oracle.hull(p).tolist(), (i, len(p))


def mixed_parts(seed):
    rng = np.random.default_rng(seed)
    parts = []
    sizes = [0, 1, 2, 3, 5, 31, 100, 999, 2047, 2048, 2049, 4097, 16384, 16385, 50000, 120001, 300000]
    for k, n in enumerate(sizes):
        fam = k % 5
        if fam == 0:
            p = W.uniform_square(n, 1 << 29, seed + k)
        elif fam == 1:
            p = W.uniform_disk(n, 2.0 ** 29, seed + k)
        elif fam == 2:
            p = W.gaussian(n, 2.0 ** 26, seed + k)
        elif fam == 3:
            p = W.near_circle(n, 2.0 ** 18, seed + k)
        else:
            p = rng.integers(-3, 4, size=(n, 2)).astype(np.int32)
        parts.append(p)
    parts.append(np.array([[7, 7]] * 5000, np.int32))            # all identical
    t = np.arange(-3000, 3000)
    parts.append(np.stack([t * 2, t * 3], axis=1).astype(np.int32))  # collinear
    parts.append(W.parabola_lattice(5000))                        # all vertices
    return parts


def test_mixed_batch(ctx):
    parts = mixed_parts(3)
    o, oo = run_batch(ctx, parts)
    check(parts, o, oo)


def test_single_and_empty_batch(ctx):
    parts = [W.uniform_disk(77777, 1e6, 5)]
    check(parts, *run_batch(ctx, parts))
    o, oo = run_batch(ctx, [])
    assert oo.tolist() == [0]


def test_uneven_batch_generator(ctx):
    pts, offs, fam = W.batch(b=300, seed=11, cap=2e7, lo=1e3, hi=3e5)
    parts = [pts[offs[i]:offs[i + 1]] for i in range(len(offs) - 1)]
    o, oo = run_batch(ctx, parts)
    check(parts, o, oo)


def test_batch_repeat_deterministic(ctx):
    parts = mixed_parts(9)
    a = run_batch(ctx, parts)
    for _ in range(3):
        b = run_batch(ctx, parts)
        assert np.array_equal(a[0][:a[1][-1]], b[0][:b[1][-1]]) and np.array_equal(a[1], b[1])


def test_batch_capacity_error(ctx, hull_lib):
    parts = [W.uniform_disk(5000, 1e6, 1), W.uniform_square(5000, 1000, 2)]
    total = sum(len(oracle.hull(p)) for p in parts)
    with pytest.raises(hull_lib.HullError) as e:
        run_batch(ctx, parts, cap=total - 1)
    assert e.value.code == hull_lib.HULL_ECAPACITY


def test_batch_range_error(ctx, hull_lib):
    lim = 1 << 29
    parts = [W.uniform_square(100, 10, 1), np.array([[0, 0], [lim + 1, 5]], np.int32)]
    with pytest.raises(hull_lib.HullError) as e:
        run_batch(ctx, parts)
    assert e.value.code == hull_lib.HULL_ERANGE


def test_batch_autotune(hull_lib, tmp_path):
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    os.environ["GBHULL_AUTOTUNE_CACHE"] = str(tmp_path / "tune.json")
    try:
        parts = mixed_parts(21)
        with hull_lib.Context(0, autotune=True) as c:
            check(parts, *run_batch(c, parts))
        assert (tmp_path / "tune.json").exists()
        txt = (tmp_path / "tune.json").read_text()
        assert "batched_small" in txt and "batched_large" in txt
        with hull_lib.Context(0, autotune=True) as c:      # reads the cache
            check(parts, *run_batch(c, parts))
    finally:
        del os.environ["GBHULL_AUTOTUNE_CACHE"]


def test_batch_learned_exact_and_discards_more(hull_lib):
    """The learned polygon inside the batched kernel: exact hulls, and it
    never discards less than the quadrilateral.  The three 300,000-point
    instances are above the size from which the batched kernel runs the
    proposal; the smaller ones take the quadrilateral."""
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from oracle import mlp as OM
    from paper_1508_05931_gb300 import learned as L
    parts = [L.instance(k % 3, 20000 + 997 * k, 300 + k) for k in range(24)] + mixed_parts(5)
    parts += [L.instance(k, 300_000, 400 + k) for k in range(3)]
    with hull_lib.Context(0, proposal=1) as c:
        c.mlp_set_params(OM.init_params(11))
        check(parts, *run_batch(c, parts))
        c.mlp_set_params(np.zeros(OM.N_PARAMS, np.float32))
        check(parts, *run_batch(c, parts))


def test_full_size_batch_sampled(hull_lib, tmp_path, monkeypatch):
    """The 4,096-instance batch at its full size (2.5e8 points, the bench's
    workload and launch configuration: one call, autotuned): the hulls of a
    seeded sample of instances, the largest and the smallest among them,
    computed one by one by the oracle, and every instance's hull size within
    its own points."""
    monkeypatch.setenv("GBHULL_AUTOTUNE_CACHE", str(tmp_path / "autotune.json"))
    pts, offs, fam = W.batch()
    dp = torch.as_tensor(pts).cuda()
    with hull_lib.Context(0, autotune=True) as c:
        o, oo = c.compute_batched(dp, torch.as_tensor(offs).cuda())
    o, oo = o.cpu().numpy(), oo.cpu().numpy()
    sizes = np.diff(offs)
    assert len(oo) == len(offs) and oo[0] == 0 and (np.diff(oo) >= 1).all()
    assert (np.diff(oo) <= sizes).all()
    rng = np.random.default_rng(77)
    pick = set(rng.choice(len(sizes), size=40, replace=False).tolist())
    pick |= {int(np.argmax(sizes)), int(np.argmin(sizes))}
    for i in sorted(pick):
        p = pts[offs[i]:offs[i + 1]]
        assert o[oo[i]:oo[i + 1]].tolist() == oracle.hull(p).tolist(), (i, len(p), int(fam[i]))


def sort_path_parts():
    """Instances for every branch of the batched sort: survivors above both
    block sizes' shared-memory capacities in bins that fit (the sort by
    groups of bins), a bin above both capacities (16,000 copies of the
    leftmost point: the radix fallback), survivors between the capacities, a
    witness bin above the per-warp limit (3,000 copies of the leftmost
    point), and mid-sized bins (near-circle sets)."""
    rng = np.random.default_rng(41)
    crowd = np.concatenate([np.tile(np.array([[-1000, 0]], np.int32), (3000, 1)),
                            rng.integers(-500, 501, size=(2000, 2)).astype(np.int32)])
    crowd = crowd[rng.permutation(len(crowd))]
    big = np.concatenate([np.tile(np.array([[-100000, 7]], np.int32), (16000, 1)),
                          W.near_circle(4000, 2.0 ** 16, 46)])
    big = big[rng.permutation(len(big))]
    return [W.parabola_lattice(20000), W.parabola_lattice(5000), crowd, big,
            W.near_circle(30000, 2.0 ** 20, 43), W.near_circle(9000, 2.0 ** 16, 44),
            W.uniform_disk(200000, 2.0 ** 28, 45)]


@pytest.mark.parametrize("block", [256, 512])
def test_batch_sort_paths_both_block_sizes(hull_lib, tmp_path, monkeypatch, block):
    import re
    cache = tmp_path / "tune.json"
    monkeypatch.setenv("GBHULL_AUTOTUNE_CACHE", str(cache))
    parts = sort_path_parts()
    with hull_lib.Context(0, autotune=True) as c:        # writes the cache for this device
        run_batch(c, parts)
    cache.write_text(re.sub(r'(batched_(?:small|large|seg_block)": )\d+', r"\g<1>%d" % block, cache.read_text()))
    with hull_lib.Context(0, autotune=True) as c:        # both buckets at the forced block size
        check(parts, *run_batch(c, parts))


def seg_parts(seed):
    """Instances of the segmented path (65,536 points or more at the default
    boundary): whole and ragged 16,384-point tiles, every family, degenerate
    sets, one with more survivors than the shared-memory sort holds, one
    whose duplicated vertex needs the radix fallback, and a few small
    instances so that every size bucket runs in the same call."""
    parts = []
    sizes = [65536, 65537, 81919, 98304, 131071, 250001]
    for k, n in enumerate(sizes):
        fam = k % 4
        if fam == 0:
            parts.append(W.uniform_square(n, 1 << 29, seed + k))
        elif fam == 1:
            parts.append(W.uniform_disk(n, 2.0 ** 29, seed + k))
        elif fam == 2:
            parts.append(W.gaussian(n, 2.0 ** 26, seed + k))
        else:
            parts.append(W.near_circle(n, 2.0 ** 22, seed + k))
    parts.append(np.array([[-5, 9]] * 70000, np.int32))                  # all identical
    t = np.arange(-40000, 40000)
    parts.append(np.stack([t, -2 * t], axis=1).astype(np.int32))         # collinear
    parts.append(W.filled_grid(300, 300, -150, -150))                    # 4 corners
    parts.append(W.near_circle(150000, 2.0 ** 20, seed + 50))            # many survivors
    # A hull vertex with 16,000 copies spread over every tile: one witness
    # bin above both shared-memory capacities (the radix fallback), where
    # the smallest of the copies' indices must come out.
    top = np.concatenate([np.tile(np.array([[3, 1 << 20]], np.int32), (16000, 1)),
                          W.uniform_disk(60000, 2.0 ** 19, seed + 70)])
    parts.append(top[np.random.default_rng(seed + 71).permutation(len(top))])
    parts += [W.uniform_disk(5, 100, seed + 60), W.uniform_square(20000, 1 << 20, seed + 61)]
    return parts


def test_segmented_path(ctx):
    parts = seg_parts(31)
    check(parts, *run_batch(ctx, parts))


def test_segmented_largest_instance(ctx, hull_lib):
    """An instance of the largest size the batched call accepts (129 tiles),
    beside a small one."""
    n = int(hull_lib.hull_batched_max_instance())
    parts = [W.uniform_disk(n, 2.0 ** 29, 71), W.uniform_square(3000, 1000, 72)]
    check(parts, *run_batch(ctx, parts))


def test_segmented_range_error(ctx, hull_lib):
    """A point out of range inside a segmented instance fails the call with
    HULL_ERANGE; the next call on the context is exact."""
    bad = W.uniform_square(70000, 1 << 20, 81).copy()
    bad[40000] = [(1 << 29) + 1, 0]
    with pytest.raises(hull_lib.HullError) as e:
        run_batch(ctx, [W.uniform_square(100, 10, 1), bad])
    assert e.value.code == hull_lib.HULL_ERANGE
    parts = seg_parts(83)
    check(parts, *run_batch(ctx, parts))


@pytest.mark.parametrize("seg_min", [1, 16385, 32768, 131072, 524288, 1 << 30])
def test_segmented_boundary_choices(hull_lib, seg_min):
    """Boundaries of the segmented path set by the caller
    (hull_config.batched_seg_min): the same instances move between the
    segmented and the one-block paths (from 1 every non-empty instance takes
    it, the degenerate ones of one, two and three points included; from
    16,385 every instance above the small bucket, and an all-vertex instance
    of 40,001 points sorts by groups after the gather; from 2^30 none)."""
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    parts = seg_parts(91) + mixed_parts(92) + [W.parabola_lattice(20000)]
    with hull_lib.Context(0, batched_seg_min=seg_min) as c:
        check(parts, *run_batch(c, parts))


def test_segmented_boundary_from_autotune_cache(hull_lib, tmp_path, monkeypatch):
    """The autotuner times the boundaries and caches its choice beside the
    block sizes; a boundary written into the cache is used by the next
    context."""
    import re
    cache = tmp_path / "tune.json"
    monkeypatch.setenv("GBHULL_AUTOTUNE_CACHE", str(cache))
    parts = seg_parts(93) + mixed_parts(94)
    with hull_lib.Context(0, autotune=True) as c:        # writes the cache for this device
        check(parts, *run_batch(c, parts))
    txt = cache.read_text()
    assert "batched_seg_min" in txt and "batched_seg_block" in txt
    cache.write_text(re.sub(r'(batched_seg_min": )\d+', r"\g<1>32768", txt))
    with hull_lib.Context(0, autotune=True) as c:
        check(parts, *run_batch(c, parts))
