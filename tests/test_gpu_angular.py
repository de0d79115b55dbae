"""Parity of the angular front (the paper's sort by angle about P_miny,
P_longest and Figure 2's forward and backward walks), called through the C
ABI, against the oracle on the same seeded inputs: the order, the position
of P_longest and every keep flag, element by element (integer work:
bit-exact)."""
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


def _check(ctx, xy):
    xy = np.ascontiguousarray(np.asarray(xy, dtype=np.int32).reshape(-1, 2))
    order, keep, l = ctx.stage_angular(torch.as_tensor(xy).cuda())
    st = oracle.angular_stages(xy)
    got = order.cpu().numpy()
    assert got.tolist() == st["order"].tolist()
    assert l == st["l_pos"]
    assert keep.cpu().numpy().tolist() == st["kept"].tolist()
    return st


def _lattice_dups():
    return np.random.default_rng(41).integers(-6, 7, size=(50_000, 2)).astype(np.int32)


def _extreme_coords():
    rng = np.random.default_rng(41)
    rng.integers(-6, 7, size=(50_000, 2))          # the lattice's draw comes first in the same stream
    return rng.integers(-(1 << 29), (1 << 29) + 1, size=(100_000, 2)).astype(np.int32)


FAMILIES = {
    "square_200k": lambda: W.uniform_square(200_000, 1 << 29, 42),
    "disk_300k": lambda: W.uniform_disk(300_000, float(1 << 29), 43),
    "near_circle_100k": lambda: W.near_circle(100_000, float(1 << 28), 44),
    "gaussian_200k": lambda: W.gaussian(200_000, float(1 << 26), 45),
    "clusters_200k": lambda: W.gaussian_clusters(200_000, 46),
    "aniso_100k": lambda: W.anisotropic_gaussian(100_000, 47),
    "grid": lambda: W.filled_grid(300, 200, -17, 5),
    "lattice_dups": _lattice_dups,
    "extreme_coords": _extreme_coords,
    "collinear": lambda: np.stack([3 * np.arange(5000) - 9000, -2 * np.arange(5000) + 7], 1).astype(np.int32),
    "vertical": lambda: np.stack([np.zeros(3000, np.int64) + 5, np.arange(3000)], 1).astype(np.int32),
    "horizontal": lambda: np.stack([np.arange(3000), np.zeros(3000, np.int64) - 4], 1).astype(np.int32),
}


@pytest.mark.parametrize("name", list(FAMILIES))
def test_angular_front_parity(ctx, name):
    _check(ctx, FAMILIES[name]())


@pytest.mark.parametrize("n", [1, 2, 3, 5, 2047, 2048, 2049, 4097, 65537])
def test_angular_front_ragged_sizes(ctx, n):
    # sizes around the walks' tile of 2048 positions, every point surviving
    # the first round (a ring), plus uniform points
    _check(ctx, W.near_circle(n, float(1 << 20), 50 + n))
    _check(ctx, W.uniform_disk(n, float(1 << 20), 60 + n))


def test_angular_front_degenerate(ctx):
    st = _check(ctx, np.full((100, 2), 7, np.int32))                    # one distinct point
    assert st["l_pos"] == -1
    _check(ctx, np.array([[3, 4]], np.int32))
    _check(ctx, np.array([[0, 0], [5, 0]], np.int32))                   # angle 0 only
    _check(ctx, np.array([[0, 0], [-5, 3], [5, 3]], np.int32))
    ring = W.near_circle(4000, float(1 << 24), 70)
    _check(ctx, np.concatenate([ring, ring, ring[:100]]))               # every point duplicated


def test_angular_front_large(ctx):
    # a few hundred walk tiles: 2M disk points, about 0.7M first-round survivors
    _check(ctx, W.uniform_disk(2_000_000, float(1 << 29), 80))


def test_angular_front_hand_trace(ctx):
    import json
    import os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "angular_second_round_trace.json")))
    xy = np.array(g["points"], dtype=np.int32)
    st = _check(ctx, xy)
    names = g["names"]
    assert [names[i] for i in st["survivors"]] == [n for n in g["expected_kept"] if n not in g["expected_first_round_removed"]]


def test_angular_front_farey_directions(ctx):
    # directions whose slopes differ by 1 / (F_k F_{k+1}) (consecutive
    # Fibonacci ratios, close to the key's 2^-60 bound), in all four 45-degree
    # sectors, exact sector boundaries, and equal directions at several
    # lengths; anchor (0, -2^29), so |dx| <= 2^29 and dy <= 2^30
    F = [0, 1]
    while len(F) < 46:
        F.append(F[-1] + F[-2])
    dirs = []
    for k in (40, 41, 42, 43):
        a, b, c = F[k - 1], F[k], F[k + 1]
        dirs += [(b, a), (a, F[k - 2]), (a, b), (b, c), (-a, b), (-b, c), (-b, a), (-a, F[k - 2])]
    dirs += [(5000, 0), (1000, 1000), (999, 1000), (1000, 999), (0, 5000), (-7000, 7000), (-6999, 7000),
             (-5000, 1), (1 << 29, 1), (-(1 << 29), 1), (1 << 29, 1 << 30), (-(1 << 29), 1 << 30)]
    dirs += [(3 * s, 2 * s) for s in (1, 2, 5, 40)] + [(-2 * s, 3 * s) for s in (1, 3, 7)]
    xy = np.array([(0, -(1 << 29))] + [(dx, dy - (1 << 29)) for dx, dy in dirs], dtype=np.int64)
    assert np.abs(xy).max() <= 1 << 29
    _check(ctx, xy.astype(np.int32))


def _lexrot(xy, h):
    """The cycle h rotated to begin at its lexicographically smallest point."""
    h = [int(v) for v in h]
    if not h:
        return h
    k = min(range(len(h)), key=lambda i: (int(xy[h[i], 0]), int(xy[h[i], 1])))
    return h[k:] + h[:k]


def _check_hull(ctx, xy):
    xy = np.ascontiguousarray(np.asarray(xy, dtype=np.int32).reshape(-1, 2))
    got = ctx.compute_angular(torch.as_tensor(xy).cuda()).cpu().numpy().tolist()
    st = oracle.angular_stages(xy)
    assert got == _lexrot(xy, st["hull"])                   # Graham's scan over the oracle's survivors
    ref = oracle.hull(xy)
    assert sorted(map(tuple, xy[got].tolist())) == sorted(map(tuple, xy[ref].tolist()))


@pytest.mark.parametrize("name", ["square_200k", "disk_300k", "near_circle_100k", "clusters_200k", "grid",
                                  "lattice_dups", "extreme_coords", "collinear", "vertical", "horizontal"])
def test_angular_hull_parity(ctx, name):
    _check_hull(ctx, FAMILIES[name]())


def test_angular_hull_small_and_degenerate(ctx):
    for xy in (np.full((9, 2), 3, np.int32), np.array([[1, 2]], np.int32), np.array([[0, 0], [5, 0]], np.int32),
               np.array([[0, 0], [-5, 3], [5, 3]], np.int32)):
        _check_hull(ctx, xy)
    ring = W.near_circle(4000, float(1 << 24), 70)
    _check_hull(ctx, np.concatenate([ring, ring, ring[:100]]))
    for seed in range(30):
        rng = np.random.default_rng(300 + seed)
        n = int(rng.integers(1, 60))
        _check_hull(ctx, rng.integers(-4, 5, size=(n, 2)).astype(np.int32))
    assert ctx.compute_angular(torch.zeros((0, 2), dtype=torch.int32).cuda()).numel() == 0

