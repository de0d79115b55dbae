"""Pins of the learned proposal's CPU oracle (oracle/learned.py) to facts it
does not compute itself: an exact area formulation of strict insideness,
label values counted by hand on a lattice diamond, and features of point
sets built so that every bin count, bin radius and direction maximum is
known in advance.  Each pin is also run against a copy of the oracle with
a planted mistake (a non-strict inside test, a bin offset by one, a wrong
radius normaliser, a dropped baseline), and must reject it."""
import inspect
import math
import types
from fractions import Fraction

import numpy as np
import pytest

import oracle
from oracle import learned as OL


# ---- planted mistakes ---------------------------------------------------

def mutant(old, new):
    """A copy of oracle.learned whose source has `old` replaced by `new`."""
    src = inspect.getsource(OL)
    assert src.count(old) == 1, old
    mod = types.ModuleType("learned_mutant")
    exec(compile(src.replace(old, new), "learned_mutant", "exec"), mod.__dict__)
    return mod


def rejects(pin, mod):
    try:
        pin(mod)
    except AssertionError:
        return True
    return False


# ---- inside_counts: strict insideness by areas ---------------------------

def strictly_inside_by_area(p, poly):
    """p is strictly inside the convex CCW polygon iff every triangle
    (p, c_j, c_j+1) has positive area and the areas sum to the polygon's."""
    k = len(poly)
    if k < 3:
        return False
    area = sum(Fraction(int(poly[j][0]) * int(poly[(j + 1) % k][1])
                        - int(poly[(j + 1) % k][0]) * int(poly[j][1])) for j in range(k))
    tri = [(int(poly[j][0]) - int(p[0])) * (int(poly[(j + 1) % k][1]) - int(p[1]))
           - (int(poly[j][1]) - int(p[1])) * (int(poly[(j + 1) % k][0]) - int(p[0])) for j in range(k)]
    return all(t > 0 for t in tri) and sum(tri) == area


def polygon_cases():
    """Random convex polygons with even coordinates (edge midpoints are
    lattice points) and probe sets holding their corners, their edge
    midpoints and random lattice points around them."""
    rng = np.random.default_rng(17)
    cases = []
    for t in range(60):
        pts = 2 * rng.integers(-6, 7, size=(int(rng.integers(3, 12)), 2))
        h = oracle.hull(pts.astype(np.int32))
        poly = pts[h].astype(np.int64)
        mids = (poly + np.roll(poly, -1, axis=0)) // 2
        probe = np.concatenate([poly, mids, rng.integers(-14, 15, size=(40, 2))]).astype(np.int64)
        cases.append((probe, poly))
    return cases


def pin_inside_counts(mod):
    boundary_seen = 0
    for probe, poly in polygon_cases():
        want = sum(strictly_inside_by_area(p, poly) for p in probe)
        assert mod.inside_counts(probe, poly) == want
        boundary_seen += len(poly) >= 3
    assert boundary_seen > 0


def test_inside_counts_equals_area_test():
    pin_inside_counts(OL)


def test_inside_counts_pin_rejects_non_strict_test():
    assert rejects(pin_inside_counts, mutant("inside &= o > 0", "inside &= o >= 0"))


def test_inside_counts_degenerate_polygons():
    pts = np.array([[0, 0], [1, 1], [2, 2]], np.int64)
    assert OL.inside_counts(pts, np.zeros((0, 2), np.int64)) == 0
    assert OL.inside_counts(pts, np.array([[0, 0], [4, 4]])) == 0


# ---- labels: counted by hand on a lattice diamond -------------------------

def diamond(r=5, c=5):
    """Every lattice point with |x - c| + |y - c| <= r, in scan order."""
    return np.array([[x, y] for x in range(c - r, c + r + 1) for y in range(c - r, c + r + 1)
                     if abs(x - c) + abs(y - c) <= r], np.int32)


def pin_labels(mod):
    xy = diamond()                                  # 61 points: 2r^2 + 2r + 1
    n = len(xy)
    assert n == 61
    corners = [[0, 5], [5, 0], [10, 5], [5, 10]]
    # ext candidates: the 4 corners and 2 edge points (labels exactly 0),
    # (10, 10): the pentagon adds the 4 inner points of the upper-right edge;
    # (20, 5): the kite adds the 9 right-half boundary points but its corners
    ext = np.array(corners + [[7, 2], [2, 3], [10, 10], [20, 5]] + [[5, 0]] * 24, np.int32)
    lab, base = mod.labels(xy, ext)
    assert base == pytest.approx(41 / 61, abs=0)    # the interior |u| + |v| <= 4: 2*16 + 8 + 1
    want = np.zeros(32)
    want[6] = 4 / 61
    want[7] = 9 / 61
    assert np.array_equal(lab, want)


def test_labels_closed_form():
    pin_labels(OL)


def test_labels_pin_rejects_dropped_baseline():
    assert rejects(pin_labels, mutant("(inside_counts(xy, pts[h]) - base) / len(xy)",
                                      "inside_counts(xy, pts[h]) / len(xy)"))


def test_labels_pin_rejects_non_strict_inside():
    assert rejects(pin_labels, mutant("inside &= o > 0", "inside &= o >= 0"))


# ---- features: sets with known bins, radii and direction maxima ----------

def bin_centre(b):
    return -math.pi + (b + 0.5) * 2 * math.pi / 32


def built_set():
    """Points in symmetric pairs (p, -p), so the mean is exactly (0, 0);
    each at the centre angle of its bin (rounding moves the angle by about
    1e-6, the bins are 0.196 wide).  Bin b (and its opposite b + 16) holds
    counts[b] points with radii radii[b][k].  Returns (points, counts,
    max radius per bin)."""
    rng = np.random.default_rng(23)
    counts = np.zeros(32, np.int64)
    maxr = np.zeros(32)
    pts = []
    for b in range(16):
        m = int(rng.integers(0, 6)) if b % 5 else 0          # some bins stay empty
        radii = rng.integers(200_000, 3_000_000, size=m)
        for r in radii:
            x = int(round(r * math.cos(bin_centre(b))))
            y = int(round(r * math.sin(bin_centre(b))))
            pts += [[x, y], [-x, -y]]
            rr = math.hypot(x, y)
            maxr[b] = max(maxr[b], rr)
            maxr[b + 16] = max(maxr[b + 16], rr)
        counts[b] += m
        counts[b + 16] += m
    return np.array(pts, np.int32), counts, maxr


def pin_features(mod):
    xy, counts, maxr = built_set()
    n = len(xy)
    assert n <= mod.SAMPLE
    feat, dmax, idx, dots = mod.features(xy)
    assert idx.tolist() == list(range(n))               # below the sample size: every point
    assert np.array_equal(feat[:32] * n, counts.astype(np.float32))
    np.testing.assert_allclose(feat[32:], maxr / maxr.max(), rtol=2e-6, atol=0)
    # direction maxima against brute-force dot products in float64
    for j in range(32):
        a = 2 * math.pi * (j % 16) / 32
        u = (math.cos(a), math.sin(a)) if j < 16 else (-math.cos(a), -math.sin(a))
        want = max(u[0] * float(x) + u[1] * float(y) for x, y in xy)
        assert abs(dmax[j] - want) <= 1e-6 * maxr.max()


def test_features_on_built_sets():
    pin_features(OL)


def test_features_pin_rejects_bin_offset():
    assert rejects(pin_features, mutant("b = np.clip(b, 0, NB - 1)", "b = np.clip(b + 1, 0, NB - 1)"))


def test_features_pin_rejects_wrong_radius_normaliser():
    assert rejects(pin_features, mutant("maxr / mr if mr > 0", "maxr / maxr.sum() if mr > 0"))


def test_sample_indices_definition():
    """The strided sample i_k = floor(k n / S), S = min(n, SAMPLE): every
    point below the sample size, an exact stride at multiples of it."""
    assert OL.sample_indices(1000).tolist() == list(range(1000))
    s = OL.SAMPLE
    assert OL.sample_indices(3 * s).tolist() == [3 * k for k in range(s)]
    idx = OL.sample_indices(5 * s + 7).astype(np.int64)
    assert len(idx) == s and idx[0] == 0 and np.all(np.diff(idx) >= 5) and idx[-1] < 5 * s + 7
