"""End-to-end parity: hull_compute (all stages on the GPU) against the
oracle's hull by definition, bit-exact, on the paper-shaped workloads at
reduced and full size, degenerate inputs and the error paths."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1508_05931_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def sctx(hull_lib):
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    c = hull_lib.Context(0, collect_stats=True)
    yield c
    c.close()


@pytest.fixture(scope="module", params=["stats", "single_read"])
def ctx(hull_lib, request):
    """The hull tests run twice: with statistics (the two-read front, which
    counts every first-round survivor) and without (inputs of 65,536 points
    or more then take the single-read front)."""
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    c = hull_lib.Context(0, collect_stats=request.param == "stats")
    c.with_stats = request.param == "stats"
    yield c
    c.close()


def dev(a):
    if not isinstance(a, np.ndarray):
        a = np.asarray(a, dtype=np.int32).reshape(-1, 2)
    return torch.as_tensor(np.ascontiguousarray(a)).cuda()


def gpu_hull(ctx, pts):
    return ctx.compute(dev(pts)).cpu().numpy()


def test_degenerate_inputs(ctx):
    assert gpu_hull(ctx, np.zeros((0, 2), np.int32)).tolist() == []
    assert gpu_hull(ctx, [[5, 7]]).tolist() == [0]
    assert gpu_hull(ctx, [[5, 7], [1, 2]]).tolist() == [1, 0]
    assert gpu_hull(ctx, [[5, 7], [5, 7]]).tolist() == [0]
    assert gpu_hull(ctx, [[3, 3]] * 9000).tolist() == [0]
    col = np.array([[i * 2, i * 3] for i in np.random.default_rng(0).integers(-500, 500, 10000)], np.int32)
    assert gpu_hull(ctx, col).tolist() == oracle.hull(col).tolist()
    g = W.filled_grid(300, 200, -7, 9)
    assert gpu_hull(ctx, g).tolist() == oracle.hull(g).tolist()
    par = W.parabola_lattice(1 << 14)
    assert gpu_hull(ctx, par).tolist() == list(range(len(par)))
    lim = 1 << 29
    edge = np.array([[lim, -lim], [-lim, lim], [0, 1], [lim, lim], [-lim, -lim]], np.int32)
    assert gpu_hull(ctx, edge).tolist() == oracle.hull(edge).tolist()


def test_random_small_sets(ctx):
    rng = np.random.default_rng(42)
    for t in range(300):
        n = int(rng.integers(1, 3000))
        span = int(rng.choice([1, 2, 5, 100, 1 << 20, 1 << 29]))
        pts = rng.integers(-span, span + 1, size=(n, 2)).astype(np.int32)
        assert gpu_hull(ctx, pts).tolist() == oracle.hull(pts).tolist(), (t, n, span)


@pytest.mark.parametrize("n", [4095, 4096, 4097, 65536, 65537, 1_000_003])
@pytest.mark.parametrize("gen", ["square", "disk", "ring", "gauss", "clusters", "ellipse"])
def test_ragged_sizes(ctx, n, gen):
    f = {"square": lambda: W.uniform_square(n, 1 << 29, n),
         "disk": lambda: W.uniform_disk(n, 2.0 ** 29, n),
         "ring": lambda: W.near_circle(n, 2.0 ** 20, n),
         "gauss": lambda: W.gaussian(n, 2.0 ** 26, n),
         "clusters": lambda: W.gaussian_clusters(n, n),
         "ellipse": lambda: W.elliptic_disk(n, n)}[gen]
    pts = f()
    assert gpu_hull(ctx, pts).tolist() == oracle.hull(pts).tolist()


def test_small_square_config(sctx):
    ctx = sctx
    pts = W.small_square()
    h = gpu_hull(ctx, pts)
    assert h.tolist() == oracle.hull(pts).tolist()
    st = ctx.last_stats()
    stages = oracle.gscan_stages(pts)
    assert st["s"] == len(stages["keep"])
    assert st["r_lower"] == len(stages["lower"]) and st["r_upper"] == len(stages["upper"])
    assert st["ext"] == stages["ext"].tolist()


def _front_points(gen, n):
    rng = np.random.default_rng(n + len(gen))
    return {"square": lambda: W.uniform_square(n, 1 << 29, n),
            "disk": lambda: W.uniform_disk(n, 2.0 ** 29, n),
            "ring": lambda: W.near_circle(n, 2.0 ** 20, n),
            "gauss": lambda: W.gaussian(n, 2.0 ** 26, n),
            "clusters": lambda: W.gaussian_clusters(n, n),
            "ties": lambda: rng.integers(-60, 61, size=(n, 2)).astype(np.int32),
            "strip": lambda: np.stack([rng.integers(-3, 4, n), rng.integers(-(1 << 29), 1 << 29, n)],
                                      axis=1).astype(np.int32)}[gen]()


@pytest.mark.parametrize("n", [4097, 65537, 300_001, 1_000_003])
@pytest.mark.parametrize("gen", ["square", "disk", "ring", "gauss", "clusters", "ties", "strip"])
def test_fused_second_round_lists(sctx, n, gen):
    """The second round fused into the sort (Figure 2 run on every sorted
    or binned group from its prefix) keeps exactly the oracle's points, in
    the oracle's order, in both regions."""
    pts = _front_points(gen, n)
    lo, up, _ = sctx.stage_regions(dev(pts))
    ref = oracle.gscan_stages(pts)
    assert np.array_equal(lo.cpu().numpy(), ref["lower"])
    assert np.array_equal(up.cpu().numpy(), ref["upper"])


@pytest.fixture(scope="module")
def rctx(hull_lib):
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    c = hull_lib.Context(0, collect_stats=True, reverse_round=True)
    yield c
    c.close()


@pytest.mark.parametrize("n", [4097, 65537, 1_000_003])
@pytest.mark.parametrize("gen", ["square", "disk", "ring", "gauss", "clusters", "ties", "strip"])
def test_reverse_round_lists(rctx, n, gen):
    """The mirrored second round on the device keeps exactly the oracle's
    points, in order, in both regions, and the hull stays the hull."""
    pts = _front_points(gen, n)
    lo, up, _ = rctx.stage_regions(dev(pts))
    ref = oracle.gscan_stages(pts, reverse=True)
    assert np.array_equal(lo.cpu().numpy(), ref["lower"])
    assert np.array_equal(up.cpu().numpy(), ref["upper"])
    assert gpu_hull(rctx, pts).tolist() == ref["hull"].tolist()
    st = rctx.last_stats()
    assert st["r_lower"] == len(ref["lower"]) and st["r_upper"] == len(ref["upper"])


def test_reverse_round_edge_cases(rctx):
    """Degenerate inputs, the radix-pass rerun, the host entry points and a
    ring whose survivors are mostly hull vertices, all with the mirrored round."""
    for pts in (np.zeros((0, 2), np.int32), np.array([[5, 7]], np.int32), np.array([[5, 7], [1, 2]], np.int32),
                np.full((9000, 2), 3, np.int32), W.filled_grid(300, 200, -7, 9), W.parabola_lattice(1 << 12),
                np.array([[i * 2, i * 3] for i in range(-500, 500)], np.int32)):
        assert gpu_hull(rctx, pts).tolist() == oracle.hull(pts).tolist()
    rng = np.random.default_rng(9)
    few = rng.integers(-1000, 1000, size=(40, 2)).astype(np.int32)
    dup = few[rng.integers(0, 40, size=300_000)]
    assert gpu_hull(rctx, dup).tolist() == oracle.hull(dup).tolist()
    assert gpu_hull(rctx, np.full((20000, 2), 77, np.int32)).tolist() == [0]
    assert rctx.last_stats()["sort_fallback"] == 1
    ring = W.near_circle(400_000, 2.0 ** 22, 7)
    ref = oracle.gscan_stages(ring, reverse=True)
    assert rctx.compute_host(ring).tolist() == ref["hull"].tolist()
    st = rctx.last_stats()
    assert st["r_lower"] == len(ref["lower"]) and st["r_upper"] == len(ref["upper"])
    sets = [W.uniform_square(200_000, 1 << 29, 3), W.uniform_disk(100_000, 2.0 ** 29, 4)]
    for p, h in zip(sets, rctx.compute_host_multi(sets)):
        assert h.tolist() == oracle.hull(p).tolist()


@pytest.mark.parametrize("name", ["paper_square", "paper_disk", "adversarial_ring"])
def test_full_size_configs(ctx, name):
    pts = getattr(W, name)()
    t = dev(pts)
    out = torch.empty(len(pts), dtype=torch.int32, device="cuda")
    h = ctx.compute(t, out=out).cpu().numpy()
    assert h.tolist() == oracle.hull(pts).tolist()
    if ctx.with_stats:
        assert ctx.last_stats()["sort_fallback"] == 0


def test_sort_fallback_only_when_needed(sctx):
    ctx = sctx
    """The bucket sort takes the paper-shaped inputs itself; identical or
    heavily duplicated points (a bin it cannot split) are rerun on the radix
    passes, with the same hull."""
    for pts in (W.uniform_square(300_000, 1 << 29, 11), W.uniform_disk(300_000, 2.0 ** 29, 12),
                W.near_circle(400_000, 2.0 ** 28, 13)):
        assert gpu_hull(ctx, pts).tolist() == oracle.hull(pts).tolist()
        assert ctx.last_stats()["sort_fallback"] == 0
    same = np.full((20000, 2), 77, np.int32)
    assert gpu_hull(ctx, same).tolist() == [0]
    assert ctx.last_stats()["sort_fallback"] == 1
    rng = np.random.default_rng(9)
    few = rng.integers(-1000, 1000, size=(40, 2)).astype(np.int32)
    dup = few[rng.integers(0, 40, size=400_000)]
    assert gpu_hull(ctx, dup).tolist() == oracle.hull(dup).tolist()


def test_determinism_repeated(ctx):
    pts = W.uniform_disk(2_000_000, 2.0 ** 29, 77)
    t = dev(pts)
    ref = ctx.compute(t).cpu().numpy()
    for _ in range(10):
        assert np.array_equal(ctx.compute(t).cpu().numpy(), ref)


def test_unaligned_input_view(ctx):
    pts = W.uniform_square(300001, 1 << 29, 5)
    view = dev(pts)[1:]
    assert view.data_ptr() % 16 == 8
    assert ctx.compute(view).cpu().numpy().tolist() == oracle.hull(pts[1:]).tolist()


def test_device_multi_entry_point(ctx, hull_lib):
    """Several device inputs back to back with one synchronisation: every
    result equals the oracle's, including an input the bucket sort hands to
    the radix passes, an empty one and a one-point one; a too-small output
    fails that input alone with a capacity error."""
    rng = np.random.default_rng(21)
    sets = [W.uniform_square(300_000, 1 << 29, 31), W.uniform_disk(200_000, 2.0 ** 29, 32),
            np.full((20000, 2), 5, np.int32), np.zeros((0, 2), np.int32), np.array([[3, 4]], np.int32),
            rng.integers(-40, 41, size=(50_000, 2)).astype(np.int32), W.near_circle(100_000, 2.0 ** 20, 33)]
    ts = [dev(p) for p in sets]
    outs = [torch.empty(max(len(p), 1), dtype=torch.int32, device="cuda") for p in sets]
    res = ctx.compute_multi(ts, outs)
    for p, h in zip(sets, res):
        assert h.cpu().numpy().tolist() == oracle.hull(p).tolist()
    small = [torch.empty(len(p) if i != 1 else 3, dtype=torch.int32, device="cuda").fill_(-1)
             for i, p in enumerate(sets[:3])]
    with pytest.raises(hull_lib.HullError) as ei:
        ctx.compute_multi(ts[:3], small)
    assert ei.value.code == hull_lib.HULL_ECAPACITY
    assert small[0][: len(oracle.hull(sets[0]))].cpu().numpy().tolist() == oracle.hull(sets[0]).tolist()
    assert small[2][:1].cpu().numpy().tolist() == oracle.hull(sets[2]).tolist()
    assert (small[1].cpu().numpy() == -1).all()
    # With the stage events on, the same results one call at a time.
    ctx.set_profiling(True)
    try:
        res = ctx.compute_multi(ts, outs)
    finally:
        ctx.set_profiling(False)
    for p, h in zip(sets, res):
        assert h.cpu().numpy().tolist() == oracle.hull(p).tolist()


def test_device_multi_full_size_two_lanes(ctx):
    """The bench's step: the 20M square, the 20M disk and the 4M ring in one
    multi call (both lanes, at full size), each hull equal to the oracle's."""
    sets = [W.paper_square(), W.paper_disk(), W.adversarial_ring()]
    ts = [dev(p) for p in sets]
    outs = [torch.empty(len(p), dtype=torch.int32, device="cuda") for p in sets]
    for _ in range(2):
        res = ctx.compute_multi(ts, outs)
        for p, h in zip(sets, res):
            assert h.cpu().numpy().tolist() == oracle.hull(p).tolist()


def test_host_entry_point(ctx):
    pts = W.uniform_disk(500_000, 2.0 ** 29, 8)
    pinned = torch.as_tensor(pts).pin_memory()
    h = ctx.compute_host(pinned)
    assert h.tolist() == oracle.hull(pts).tolist()
    h2 = ctx.compute_host(pts)
    assert h2.tolist() == oracle.hull(pts).tolist()


def test_host_multi_entry_point(ctx, hull_lib):
    """Several host inputs in one pipelined call (the copy of input k + 1
    overlaps the hull of input k): every result equals the oracle's, for
    pinned and pageable inputs, an empty input, sizes that grow the staging
    buffers, and a capacity failure that stops the sequence."""
    sets = [W.uniform_disk(300_000, 2.0 ** 29, 21), np.zeros((0, 2), np.int32),
            W.uniform_square(1_200_000, 1 << 29, 22), W.uniform_square(7, 1 << 20, 23),
            W.uniform_disk(2_500_000, 2.0 ** 28, 24)]
    refs = [oracle.hull(p).tolist() for p in sets]
    pinned = [torch.as_tensor(p).pin_memory() for p in sets]
    got = ctx.compute_host_multi(pinned)
    assert [g.tolist() for g in got] == refs
    got = ctx.compute_host_multi(sets)
    assert [g.tolist() for g in got] == refs
    assert ctx.compute_host_multi([]) == []
    # the single-input host entry still works with the grown staging
    assert ctx.compute_host(pinned[2]).tolist() == refs[2]
    small = [np.empty(1, np.int32) for _ in sets]
    with pytest.raises(hull_lib.HullError) as ei:
        ctx.compute_host_multi(pinned, outs=small)
    assert ei.value.code == hull_lib.HULL_ECAPACITY
    assert ctx.compute_host_multi(pinned[:2])[0].tolist() == refs[0]


def test_range_error(ctx, hull_lib):
    lim = 1 << 29
    bad = np.array([[0, 0], [lim + 1, 0], [3, 4]], np.int32)
    with pytest.raises(hull_lib.HullError) as e:
        ctx.compute(dev(bad))
    assert e.value.code == hull_lib.HULL_ERANGE
    bad2 = np.array([[0, -lim - 1], [1, 1]], np.int32)
    with pytest.raises(hull_lib.HullError):
        ctx.compute(dev(bad2))
    # the context stays usable
    ok = W.uniform_square(1000, 100, 1)
    assert gpu_hull(ctx, ok).tolist() == oracle.hull(ok).tolist()


def test_capacity_error_reports_count(ctx, hull_lib):
    pts = W.uniform_disk(10000, 1e6, 3)
    ref = oracle.hull(pts)
    t = dev(pts)
    out = torch.full((len(ref) - 1,), -5, dtype=torch.int32, device="cuda")
    cnt = ctypes.c_int64()
    rc = hull_lib._lib.hull_compute(ctx.handle, ctypes.c_void_p(t.data_ptr()), len(pts),
                                    ctypes.c_void_p(out.data_ptr()), out.numel(), ctypes.byref(cnt),
                                    None)
    torch.cuda.synchronize()
    assert rc == hull_lib.HULL_ECAPACITY and cnt.value == len(ref)
    assert bool((out == -5).all())


def test_invalid_arguments(ctx, hull_lib):
    cnt = ctypes.c_int64()
    L = hull_lib._lib
    assert L.hull_compute(ctx.handle, None, 10, None, 0, ctypes.byref(cnt), None) == hull_lib.HULL_EINVAL
    assert L.hull_compute(ctx.handle, None, -1, None, 0, ctypes.byref(cnt), None) == hull_lib.HULL_EINVAL
    t = dev(np.zeros((4, 2), np.int32))
    assert L.hull_compute(ctx.handle, ctypes.c_void_p(t.data_ptr() + 4), 2, None, 0, ctypes.byref(cnt),
                          None) == hull_lib.HULL_EINVAL
    assert L.hull_compute(ctx.handle, ctypes.c_void_p(t.data_ptr()), 1 << 30, None, 0,
                          ctypes.byref(cnt), None) == hull_lib.HULL_EINVAL


def test_forced_wait_timeouts_recover(hull_lib):
    """Failure detection, injected from the host: with a spin limit of one
    iteration, every bounded device wait that is not satisfied at once gives
    up.  The radix passes look back at earlier tiles (4M keys, thousands of
    tiles on a few hundred blocks) and the final chain of the 4M near-circle
    set crosses grid barriers over many blocks, so such waits must run out:
    at least one call has to report HULL_ETIMEOUT, every other result must be
    exact, no call may hang or trap, and a context with the normal limit must
    give the oracle's hull afterwards."""
    pts = W.near_circle(4_000_000, 2.0 ** 28, 3)
    ref = oracle.hull(pts)
    t = dev(pts)
    rng = np.random.default_rng(7)
    keys_np = rng.integers(0, 1 << 62, size=4_000_000, dtype=np.int64)
    order = np.argsort(keys_np, kind="stable")
    codes = []
    with hull_lib.Context(0, spin_limit=1) as c:
        for _ in range(3):
            try:
                h = c.compute(t).cpu().numpy()
                assert h.tolist() == ref.tolist()
                codes.append(hull_lib.HULL_OK)
            except hull_lib.HullError as e:
                assert e.code == hull_lib.HULL_ETIMEOUT
                codes.append(e.code)
            k = torch.as_tensor(keys_np).cuda()
            v = torch.arange(len(keys_np), dtype=torch.int32, device="cuda")
            try:
                c.stage_sort(k, v)
                assert v.cpu().numpy().tolist() == order.tolist()
                codes.append(hull_lib.HULL_OK)
            except hull_lib.HullError as e:
                assert e.code == hull_lib.HULL_ETIMEOUT
                codes.append(e.code)
    assert hull_lib.HULL_ETIMEOUT in codes, codes
    with hull_lib.Context(0) as c:
        assert c.compute(t).cpu().numpy().tolist() == ref.tolist()


def test_single_read_front_edge_cases(ctx):
    """Inputs of 65,536 points or more (16-byte aligned, no statistics) take
    the single-read front: the sample polygon drops the points strictly
    inside it during the extremes pass.  Its degenerate and boundary cases,
    each against the oracle: identical, collinear and two-column inputs (no
    polygon with an interior: nothing is dropped), a filled lattice whose
    sample polygon has lattice points on its edges, a thin sliver, a tight
    cluster with a sparse halo, heavy duplicates, odd sizes just above the
    threshold, and an unaligned view (the two-read front)."""
    rng = np.random.default_rng(61)
    t = np.arange(-100_000, 100_000)
    sets = {
        "identical": np.full((200_000, 2), -123, np.int32),
        "collinear": np.stack([t * 3, t * 7], axis=1).astype(np.int32),
        "two_columns": np.stack([rng.integers(0, 2, 150_000), rng.integers(-1 << 29, 1 << 29, 150_000)],
                                axis=1).astype(np.int32),
        "lattice": W.filled_grid(400, 400, -200, -150),
        "sliver": np.stack([t, t // 1000 + rng.integers(0, 3, t.size)], axis=1).astype(np.int32),
        "cluster_halo": np.concatenate([rng.integers(-50, 51, size=(300_000, 2)),
                                        rng.integers(-(1 << 28), 1 << 28, size=(3_000, 2))]).astype(np.int32),
        "duplicates": rng.integers(-1000, 1000, size=(60, 2)).astype(np.int32)[rng.integers(0, 60, size=400_000)],
        "odd_above": W.uniform_disk(65_537, 2.0 ** 29, 62),
        "odd_large": W.uniform_square(1_000_001, 1 << 29, 63),
    }
    for name, pts in sets.items():
        assert gpu_hull(ctx, pts).tolist() == oracle.hull(pts).tolist(), name
    pts = W.uniform_disk(300_001, 2.0 ** 29, 64)
    buf = torch.as_tensor(np.concatenate([np.zeros((1, 2), np.int32), pts])).cuda()
    view = buf[1:]
    assert view.data_ptr() % 16 == 8
    assert ctx.compute(view).cpu().numpy().tolist() == oracle.hull(pts).tolist()
