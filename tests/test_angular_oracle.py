"""Pins for the oracle of the paper's angular ordering (Section 2.1 steps 3-8
with the sort by angle of Sections 3.2-3.3): the order against exact rational
slopes and fp64 atan2, the second round's survivors against the hull's
vertices, the final hull against the hull by definition and O(n^3) brute
force, and a hand-derived trace of both walks of Figure 2 in tests/golden/.
All CPU-only."""
import importlib.util
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_1508_05931_gb300 import workloads as W

HERE = os.path.dirname(__file__)
GOLDEN = os.path.join(HERE, "golden")

_spec = importlib.util.spec_from_file_location("_pins", os.path.join(HERE, "test_oracle_pins.py"))
_pins = importlib.util.module_from_spec(_spec)
_spec.loader.exec_module(_pins)
brute_hull = _pins.brute_hull


def _orient(a, b, c):
    return (int(b[0]) - int(a[0])) * (int(c[1]) - int(a[1])) - (int(b[1]) - int(a[1])) * (int(c[0]) - int(a[0]))


def _cycle_from(coords, start):
    """The cyclic sequence `coords` rotated to begin at `start`."""
    k = coords.index(start)
    return coords[k:] + coords[:k]


def _inputs():
    yield "square", W.uniform_square(4000, 1 << 20, 31)
    yield "disk", W.uniform_disk(4000, float(1 << 20), 32)
    yield "near_circle", W.near_circle(3000, float(1 << 24), 33)
    yield "gaussian", W.gaussian(4000, float(1 << 18), 34)
    yield "clusters", W.gaussian_clusters(4000, 35)
    yield "grid", W.filled_grid(30, 20, -7, 3)
    rng = np.random.default_rng(36)
    yield "small_range", rng.integers(-6, 7, size=(2000, 2)).astype(np.int32)     # many equal angles and duplicates
    yield "extreme_coords", rng.integers(-(1 << 29), (1 << 29) + 1, size=(3000, 2)).astype(np.int32)
    yield "collinear", np.stack([3 * np.arange(400) - 500, -2 * np.arange(400) + 7], 1).astype(np.int32)
    yield "two_points", np.array([[5, 5], [-3, 5]], dtype=np.int32)
    yield "all_equal", np.full((50, 2), 9, dtype=np.int32)
    yield "single", np.array([[1, 2]], dtype=np.int32)


# ------------------------------------------------------------------ the order

def _exact_angle_key(p, o, idx):
    """The angle about o (o lowest, leftmost among the lowest) as an exact
    rational key: (half-quadrant, slope), then the squared distance, then
    the index.  dx > 0: the angle grows with dy/dx; dx = 0: pi/2; dx < 0:
    the angle grows as dy/|dx| falls, i.e. with dy/dx."""
    dx, dy = int(p[0]) - int(o[0]), int(p[1]) - int(o[1])
    if dx > 0:
        q = (0, Fraction(dy, dx))
    elif dx == 0:
        q = (1, Fraction(0))
    else:
        q = (2, Fraction(dy, dx))
    return q + (dx * dx + dy * dy, idx)


@pytest.mark.parametrize("name,xy", list(_inputs()), ids=[n for n, _ in _inputs()])
def test_angular_order_is_the_exact_angle_order(name, xy):
    xy = np.ascontiguousarray(xy, dtype=np.int32)
    anchor = int(oracle.extremes(xy)[2])
    o = xy[anchor]
    assert all((int(p[1]), int(p[0])) >= (int(o[1]), int(o[0])) for p in xy)       # lowest, then leftmost
    idx = np.arange(len(xy))
    got = oracle.angular_sort(xy, idx, anchor).tolist()
    rest = [i for i in idx.tolist() if (xy[i, 0], xy[i, 1]) != (o[0], o[1])]
    want = sorted(rest, key=lambda i: _exact_angle_key(xy[i], o, i))
    assert got == want


def test_angular_order_matches_atan2_where_angles_are_apart():
    rng = np.random.default_rng(37)
    xy = rng.integers(-(1 << 20), 1 << 20, size=(3000, 2)).astype(np.int32)
    anchor = int(oracle.extremes(xy)[2])
    o = xy[anchor].astype(np.float64)
    got = oracle.angular_sort(xy, np.arange(len(xy)), anchor)
    ang = np.arctan2(xy[got, 1] - o[1], xy[got, 0] - o[0])
    assert np.all(ang >= 0.0) and np.all(ang < math.pi)
    d = np.diff(ang)
    far = np.abs(d) > 1e-12              # pairs fp64 separates for sure
    assert far.sum() > 0.99 * len(d)
    assert np.all(d[far] > 0)


# ---------------------------------------------------------- round and hull

def _strict_vertices(xy):
    return {tuple(map(int, xy[i])) for i in oracle.hull(xy)}


@pytest.mark.parametrize("name,xy", list(_inputs()), ids=[n for n, _ in _inputs()])
def test_angular_pipeline_hull_is_the_hull(name, xy):
    xy = np.ascontiguousarray(xy, dtype=np.int32)
    st = oracle.angular_stages(xy)
    got = [tuple(map(int, xy[i])) for i in st["hull"]]
    ref = [tuple(map(int, xy[i])) for i in oracle.hull(xy)]
    assert len(got) == len(ref) and set(got) == set(ref), name
    if len(ref) > 2:
        assert got == _cycle_from(ref, got[0]), name       # the same counter-clockwise cycle
    # the anchor starts the hull; every reported index carries its vertex
    assert st["hull"][0] == st["anchor"]
    # the second round keeps every strict vertex
    surv = {tuple(map(int, xy[i])) for i in st["survivors"]}
    assert _strict_vertices(xy) <= surv, name
    # and discards only first-round survivors' interior points
    assert set(st["survivors"].tolist()) <= set(st["order"].tolist())


@pytest.mark.parametrize("seed", range(40))
def test_angular_pipeline_vs_brute_force(seed):
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(1, 40))
    span = int(rng.choice([3, 10, 1000]))
    xy = rng.integers(-span, span + 1, size=(n, 2)).astype(np.int32)
    st = oracle.angular_stages(xy)
    got = [tuple(map(int, xy[i])) for i in st["hull"]]
    ref = [tuple(map(int, xy[i])) for i in brute_hull(xy)]
    assert set(got) == set(ref) and len(got) == len(ref)
    if len(ref) > 2:
        assert got == _cycle_from(ref, got[0])


def test_second_round_without_first_round_keeps_the_vertices():
    # the walks on their own (every point in angular order, no quadrilateral)
    xy = W.uniform_disk(5000, float(1 << 20), 38)
    anchor = int(oracle.extremes(xy)[2])
    order = np.concatenate([[anchor], oracle.angular_sort(xy, np.arange(len(xy)), anchor)])
    kept, l = oracle.angular_second_round(xy, order)
    o, pl = xy[anchor], xy[order[l]]
    d = ((xy[order, 0].astype(np.int64) - o[0]) ** 2 + (xy[order, 1].astype(np.int64) - o[1]) ** 2)
    assert d[l] == d.max() and np.argmax(d) == l                     # P_l: the first farthest point
    assert kept[0] and kept[l] and kept[-1]
    surv = {tuple(map(int, xy[i])) for i in order[kept]}
    assert _strict_vertices(xy) <= surv
    assert kept.sum() < 0.1 * len(order)
    # the two regions: before P_l right of P_0 -> P_l or on it, after P_l left or on it
    assert all(_orient(o, pl, xy[i]) <= 0 for i in order[1:l])
    assert all(_orient(o, pl, xy[i]) >= 0 for i in order[l + 1:])


def test_longest_is_the_first_of_equally_far_points():
    # hand-made: about P_0 = (0, 0) the points (5, 0), (3, 4), (0, 5) are all
    # at squared distance 25, (1, 1) at 2; angular order (5,0) 0 deg, (1,1)
    # 45 deg, (3,4) 53 deg, (0,5) 90 deg; P_l is the first of the three
    xy = np.array([[0, 5], [1, 1], [0, 0], [3, 4], [5, 0]], dtype=np.int32)
    anchor = int(oracle.extremes(xy)[2])
    assert anchor == 2
    seq = np.concatenate([[anchor], oracle.angular_sort(xy, np.arange(5), anchor)])
    assert seq.tolist() == [2, 4, 1, 3, 0]
    kept, l = oracle.angular_second_round(xy, seq)
    assert l == 1
    # forward walk empty; backward from (0,5): (3,4) is left of (0,5) -> (5,0)
    # (orient = 5*(-1) - (-5)*3 = 10 > 0), kept; (1,1) right of (3,4) -> (5,0)
    # (orient = 2*(-3) - (-4)*(-2) = -14 <= 0), interior
    assert seq[kept].tolist() == [2, 4, 3, 0]


def test_degenerate_lists():
    xy = np.array([[0, 0], [4, 0]], dtype=np.int32)
    kept, l = oracle.angular_second_round(xy, np.array([0, 1]))
    assert l == 1 and kept.tolist() == [True, True]
    kept, l = oracle.angular_second_round(xy, np.array([0]))
    assert l == -1 and kept.tolist() == [True]
    st = oracle.angular_stages(np.zeros((0, 2), np.int32))
    assert st["hull"].size == 0
    st = oracle.angular_stages(np.full((7, 2), 3, np.int32))
    assert st["hull"].tolist() == [0]


# ------------------------------------------------------------- golden trace

def test_hand_derived_trace():
    g = json.load(open(os.path.join(GOLDEN, "angular_second_round_trace.json")))
    names = g["names"]
    xy = np.array(g["points"], dtype=np.int32)
    at = {n: i for i, n in enumerate(names)}
    anchor = int(oracle.extremes(xy)[2])
    assert names[anchor] == g["expected_anchor"]
    order = oracle.angular_sort(xy, np.arange(len(xy)), anchor)
    assert [names[i] for i in order] == g["expected_angular_order"]
    seq = np.concatenate([[anchor], order])
    kept, l = oracle.angular_second_round(xy, seq)
    assert names[seq[l]] == g["expected_longest"]
    assert [names[i] for i in seq[kept]] == g["expected_kept"]
    hull = oracle.graham(xy, seq[kept])
    assert [names[i] for i in hull] == g["expected_hull_ccw"]
    st = oracle.angular_stages(xy)
    removed = sorted(set(range(len(xy))) - set(st["keep"].tolist()))
    assert sorted(names[i] for i in removed) == sorted(g["expected_first_round_removed"])
    assert [names[i] for i in st["hull"]] == g["expected_hull_ccw"]
    assert at["P0"] == anchor
