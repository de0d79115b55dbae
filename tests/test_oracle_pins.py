"""Pins for the CPU oracle: each check ties an oracle function to something
other than itself -- O(n^3) brute force, closed forms, invariants, a library
routine, exact rational geometry, statistics the geometry fixes, and the
hand-derived Figure 2 trace in tests/golden/.  All CPU-only."""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_1508_05931_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- brute force

def brute_hull(pts):
    """Hull by O(n^3) edge enumeration, independent of any chain algorithm.

    A directed pair (i, j) of distinct unique points is a hull edge iff every
    point k has orient(i, j, k) >= 0 and every k with orient == 0 lies in the
    closed segment [i, j].  Edges are chained counter-clockwise from the
    lexicographic minimum.  Duplicates keep the smallest index."""
    pts = np.asarray(pts, dtype=np.int64).reshape(-1, 2)
    n = len(pts)
    if n == 0:
        return []
    first = {}
    for i, (x, y) in enumerate(pts.tolist()):
        first.setdefault((x, y), i)
    uniq = sorted(first.items())                 # ((x, y), idx) lexicographic
    P = np.array([u[0] for u in uniq], dtype=np.int64)
    ids = [u[1] for u in uniq]
    m = len(P)
    if m == 1:
        return [ids[0]]
    d = P[None, :, :] - P[:, None, :]            # d[i, j] = P[j] - P[i]
    # o[i, j, k] = (P[j] - P[i]) x (P[k] - P[i])
    o = d[:, :, None, 0] * d[:, None, :, 1] - d[:, :, None, 1] * d[:, None, :, 0]
    dot = (d[:, :, None, 0] * d[:, None, :, 0] + d[:, :, None, 1] * d[:, None, :, 1])
    len2 = (d[:, :, 0] ** 2 + d[:, :, 1] ** 2)[:, :, None]
    inseg = (dot >= 0) & (dot <= len2)
    edge = np.all((o > 0) | ((o == 0) & inseg), axis=2)
    np.fill_diagonal(edge, False)
    out = [0]
    cur = 0
    for _ in range(m + 1):
        nxt = np.nonzero(edge[cur])[0]
        assert len(nxt) == 1, "brute force: vertex with %d outgoing edges" % len(nxt)
        cur = int(nxt[0])
        if cur == 0:
            break
        out.append(cur)
    return [ids[v] for v in out]


def rand_tiny(rng, n, span):
    return rng.integers(-span, span + 1, size=(n, 2)).astype(np.int32)


def test_brute_force_itself_on_square():
    pts = [[0, 0], [2, 0], [2, 2], [0, 2], [1, 1], [1, 0]]
    assert brute_hull(pts) == [0, 1, 2, 3]


@pytest.mark.parametrize("span", [2, 4, 100, 1 << 29])
def test_hull_matches_brute_force(span):
    rng = np.random.default_rng(1000 + span % 997)
    for trial in range(400):
        n = int(rng.integers(1, 48))
        pts = rand_tiny(rng, n, span)
        if trial % 5 == 0:                       # heavy duplicates
            pts[rng.integers(0, n, n // 2)] = pts[rng.integers(0, n)]
        if trial % 7 == 0:                       # collinear run
            t = rng.integers(-3, 4, size=n)
            pts = np.stack([t * 3, t * 2 + 1], axis=1).astype(np.int32)
        assert oracle.hull(pts).tolist() == brute_hull(pts), (span, trial, pts.tolist())


# ---------------------------------------------------------------- closed forms

def test_closed_form_parabola_lattice():
    k = 1 << 14
    pts = W.parabola_lattice(k)
    h = oracle.hull(pts)
    assert h.tolist() == list(range(2 * k + 1))


def test_closed_form_filled_grid():
    pts = W.filled_grid(37, 23, x0=-5, y0=11)
    h = oracle.hull(pts)
    xy = pts[h].tolist()
    assert xy == [[-5, 11], [31, 11], [31, 33], [-5, 33]]


def test_degenerate_sizes():
    assert oracle.hull(np.zeros((0, 2), np.int32)).tolist() == []
    assert oracle.hull([[5, 7]]).tolist() == [0]
    assert oracle.hull([[5, 7], [1, 2]]).tolist() == [1, 0]
    assert oracle.hull([[5, 7], [5, 7]]).tolist() == [0]
    assert oracle.hull([[3, 3]] * 9).tolist() == [0]
    col = [[i * 2, i * 3] for i in (4, -1, 7, 2, 7, -1, 0)]
    assert oracle.hull(col).tolist() == [1, 2]


def test_range_check():
    lim = 1 << 29
    assert oracle.hull([[lim, -lim], [-lim, lim], [0, 1]]).tolist() == [1, 0, 2]
    with pytest.raises(ValueError):
        oracle.hull([[lim + 1, 0], [0, 0]])
    with pytest.raises(ValueError):
        oracle.hull([[0, 0], [0, -lim - 1]])


def test_metamorphic_permutation_rotation_translation():
    rng = np.random.default_rng(7)
    pts = W.uniform_disk(3000, 1000.0, 11)
    h = oracle.hull(pts)
    base = sorted(map(tuple, pts[h].tolist()))
    perm = rng.permutation(len(pts))
    h2 = oracle.hull(pts[perm])
    assert sorted(map(tuple, pts[perm][h2].tolist())) == base
    rot = np.stack([-pts[:, 1], pts[:, 0]], axis=1)
    h3 = oracle.hull(rot)
    assert sorted(map(tuple, pts[h3].tolist())) == base   # same vertex set
    tr = pts + np.array([12345, -999], np.int32)
    assert oracle.hull(tr).tolist() == h.tolist()


def check_invariants(pts, h):
    pts = np.asarray(pts, dtype=np.int64)
    hv = pts[h]
    k = len(h)
    # starts at the lexicographic minimum, smallest index among duplicates
    lex = np.lexsort((np.arange(len(pts)), pts[:, 1], pts[:, 0]))
    assert h[0] == lex[0]
    if k <= 2:
        return
    for a in range(k):
        p, q, r = hv[a], hv[(a + 1) % k], hv[(a + 2) % k]
        # every point on or left of each CCW edge
        e = q - p
        o = e[0] * (pts[:, 1] - p[1]) - e[1] * (pts[:, 0] - p[0])
        assert np.all(o >= 0)
        # strict turns: no collinear boundary points reported
        assert (q - p)[0] * (r - p)[1] - (q - p)[1] * (r - p)[0] > 0
    # each vertex reported with the smallest index of its coordinates
    for v in h:
        same = np.nonzero((pts[:, 0] == pts[v, 0]) & (pts[:, 1] == pts[v, 1]))[0]
        assert v == same[0]


@pytest.mark.parametrize("gen", ["square", "disk", "ring", "gauss", "dups"])
def test_invariants_medium(gen):
    if gen == "square":
        pts = W.uniform_square(20000, 1 << 29, 3)
    elif gen == "disk":
        pts = W.uniform_disk(20000, float(1 << 29), 4)
    elif gen == "ring":
        pts = W.near_circle(20000, 3000.0, 5)
    elif gen == "gauss":
        pts = W.gaussian(20000, 1e6, 6)
    else:
        pts = W.uniform_square(20000, 30, 8)
    check_invariants(pts, oracle.hull(pts))


# ---------------------------------------------------------------- extremes

def test_extremes_match_lexsort():
    rng = np.random.default_rng(3)
    for t in range(200):
        n = int(rng.integers(1, 300))
        span = int(rng.choice([1, 3, 1000, 1 << 29]))
        pts = rand_tiny(rng, n, span)
        i = np.arange(n)
        x, y = pts[:, 0].astype(np.int64), pts[:, 1].astype(np.int64)
        exp = [np.lexsort((i, y, x))[0], np.lexsort((i, -y, -x))[0],
               np.lexsort((i, x, y))[0], np.lexsort((i, -x, -y))[0]]
        assert oracle.extremes(pts).tolist() == [int(e) for e in exp]


# ---------------------------------------------------------------- quad filter

def _strictly_inside_by_area(p, poly):
    """Exact test by areas (a formulation different from the edge signs):
    p is strictly inside a convex polygon iff the triangles (p, c_j, c_j+1)
    have positive areas summing to the polygon's area."""
    k = len(poly)
    if k < 3:
        return False
    area = sum(Fraction(int(poly[j][0]) * int(poly[(j + 1) % k][1])
                        - int(poly[(j + 1) % k][0]) * int(poly[j][1])) for j in range(k))
    tri = []
    for j in range(k):
        a, b = poly[j], poly[(j + 1) % k]
        tri.append((int(a[0]) - int(p[0])) * (int(b[1]) - int(p[1]))
                   - (int(a[1]) - int(p[1])) * (int(b[0]) - int(p[0])))
    return all(t > 0 for t in tri) and sum(tri) == area


def test_quad_filter_exact_small():
    rng = np.random.default_rng(5)
    for t in range(150):
        n = int(rng.integers(1, 80))
        pts = rand_tiny(rng, n, int(rng.choice([2, 5, 50])))
        poly = oracle.quad(pts)
        keep = set(oracle.quad_filter(pts).tolist())
        for i in range(n):
            assert (i not in keep) == _strictly_inside_by_area(pts[i], poly)
        # every strict hull vertex survives
        assert set(brute_hull(pts)) <= keep


def test_quad_corners_are_extremes_in_ccw_order():
    pts = np.array([[0, 5], [5, 0], [10, 5], [5, 10], [5, 5]], np.int32)
    assert oracle.quad(pts).tolist() == [[0, 5], [5, 0], [10, 5], [5, 10]]
    assert oracle.quad_filter(pts).tolist() == [0, 1, 2, 3]
    # an axis-aligned grid degenerates to two corners: nothing is discarded
    g = W.filled_grid(5, 5)
    assert len(oracle.quad(g)) == 2
    assert len(oracle.quad_filter(g)) == 25


def test_quad_filter_statistics():
    """Uniform square: the four corner triangles have expected total area 1/2
    of the square; uniform disk: the quad tends to the inscribed square, so
    1 - 2/pi of the points survive."""
    fr = [len(oracle.quad_filter(W.uniform_square(20000, 1 << 29, s))) / 20000 for s in range(200)]
    assert abs(np.mean(fr) - 0.5) < 0.03
    d = W.uniform_disk(400000, float(1 << 29), 9)
    assert abs(len(oracle.quad_filter(d)) / len(d) - (1 - 2 / math.pi)) < 0.01


# ---------------------------------------------------------------- sort

def test_sort_survivors_is_stable_lexicographic():
    pts = np.array([[3, 1], [1, 2], [3, 1], [1, 1], [2, 9], [1, 2]], np.int32)
    assert oracle.sort_survivors(pts, [0, 1, 2, 3, 4, 5]).tolist() == [3, 1, 5, 4, 0, 2]
    assert oracle.sort_survivors(pts, [5, 2, 0]).tolist() == [5, 0, 2]


# ---------------------------------------------------------------- second round

def _golden_trace():
    with open(os.path.join(GOLDEN, "second_round_trace.json")) as f:
        g = json.load(f)
    names, P, perm = g["names"], g["points"], g["index_permutation"]
    pts = np.zeros((len(P), 2), np.int32)
    for k, j in enumerate(perm):
        pts[j] = P[k]
    name_of = {perm[k]: names[k] for k in range(len(names))}
    return g, pts, name_of


def test_second_round_golden_trace():
    g, pts, name_of = _golden_trace()
    srt = oracle.sort_survivors(pts, np.arange(len(pts)))
    lo, up, lpos = oracle.second_round(pts, srt)
    assert [name_of[i] for i in lo] == g["expected_lower_kept"]
    assert [name_of[i] for i in up] == g["expected_upper_kept"]
    assert name_of[int(srt[lpos])] == "Pl"
    assert [name_of[i] for i in oracle.gscan_stages(pts)["hull"]] == g["expected_hull_ccw"]
    assert [name_of[i] for i in oracle.hull(pts)] == g["expected_hull_ccw"]


def _in_closed_triangle(p, a, b, c):
    def o(u, v, w):
        return (int(v[0]) - int(u[0])) * (int(w[1]) - int(u[1])) - (int(v[1]) - int(u[1])) * (int(w[0]) - int(u[0]))
    s1, s2, s3 = o(a, b, p), o(b, c, p), o(c, a, p)
    return (s1 >= 0 and s2 >= 0 and s3 >= 0) or (s1 <= 0 and s2 <= 0 and s3 <= 0)


def test_second_round_is_safe_with_witnesses():
    """Section 2.2.2: a discarded point lies in a triangle spanned by kept
    input points (P_0, an earlier kept point of its region, P_l) or is a
    duplicate/on the dividing line; every strict hull vertex survives."""
    rng = np.random.default_rng(11)
    for t in range(120):
        n = int(rng.integers(3, 60))
        pts = rand_tiny(rng, n, int(rng.choice([3, 8, 1000])))
        srt = oracle.sort_survivors(pts, np.arange(n))
        lo, up, lpos = oracle.second_round(pts, srt)
        hv = set(brute_hull(pts))
        if lpos < 0:
            assert len(hv) == 1
            continue
        p0, pl = int(srt[0]), int(srt[lpos])
        assert hv <= set(lo.tolist()) | set(up.tolist()) | {p0, pl}
        kept = set(lo.tolist()) | set(up.tolist())
        for pos in range(1, len(srt)):
            i = int(srt[pos])
            if i in kept or i == pl:
                continue
            A, B, p = pts[p0], pts[pl], pts[i]
            side = (int(B[0]) - int(A[0])) * (int(p[1]) - int(A[1])) - (int(B[1]) - int(A[1])) * (int(p[0]) - int(A[0]))
            region = lo if side < 0 else up
            wit = [p0] + [int(j) for j in region if list(srt).index(j) < pos]
            assert any(_in_closed_triangle(p, A, pts[w], B) for w in wit), (t, i)


def test_second_round_chunked_golden_trace():
    """Section 3.4's chunked second round on the hand-made points of Section
    2.2.3's trace, two runs per region (tests/golden/second_round_chunked_trace.json)."""
    with open(os.path.join(GOLDEN, "second_round_chunked_trace.json")) as f:
        g = json.load(f)
    names, P, perm = g["names"], g["points"], g["index_permutation"]
    pts = np.zeros((len(P), 2), np.int32)
    for k, j in enumerate(perm):
        pts[j] = P[k]
    name_of = {perm[k]: names[k] for k in range(len(names))}
    srt = oracle.sort_survivors(pts, np.arange(len(pts)))
    lo, up, lpos = oracle.second_round_chunked(pts, srt, g["block_size"])
    assert [name_of[i] for i in lo] == g["expected_lower_kept"]
    assert [name_of[i] for i in up] == g["expected_upper_kept"]
    assert name_of[int(srt[lpos])] == "Pl"


def test_second_round_chunked_limits_and_safety():
    """One run per region is Figure 2 itself; runs of one point keep the
    whole region; any run length keeps a superset of the exact survivors
    that holds every strict hull vertex, and every point it discards lies in
    the closed triangle (P_0, P_temp, P_l) of an earlier kept point of its
    run (or P_0)."""
    rng = np.random.default_rng(51)
    for t in range(200):
        n = int(rng.integers(3, 80))
        pts = rand_tiny(rng, n, int(rng.choice([3, 8, 1000, 1 << 29])))
        srt = oracle.sort_survivors(pts, np.arange(n))
        lo, up, lpos = oracle.second_round(pts, srt)
        c1 = oracle.second_round_chunked(pts, srt, 1)
        assert c1[0].tolist() == lo.tolist() and c1[1].tolist() == up.tolist() and c1[2] == lpos
        if lpos < 0:
            continue
        p0, pl = int(srt[0]), int(srt[lpos])
        A, B = pts[p0], pts[pl]

        def side(i):
            p = pts[i]
            return (int(B[0]) - int(A[0])) * (int(p[1]) - int(A[1])) - (int(B[1]) - int(A[1])) * (int(p[0]) - int(A[0]))

        regions = ([int(i) for i in srt[1:] if side(int(i)) < 0], [int(i) for i in srt[1:] if side(int(i)) > 0])
        cn = oracle.second_round_chunked(pts, srt, n)
        assert cn[0].tolist() == regions[0] and cn[1].tolist() == regions[1]
        hv = set(brute_hull(pts))
        for bs in (2, 3, 7):
            cl, cu, _ = oracle.second_round_chunked(pts, srt, bs)
            assert set(lo.tolist()) <= set(cl.tolist()) and set(up.tolist()) <= set(cu.tolist())
            assert hv <= set(cl.tolist()) | set(cu.tolist()) | {p0, pl}
            for reg, kept in zip(regions, (set(cl.tolist()), set(cu.tolist()))):
                run = (len(reg) + bs - 1) // bs
                for k, i in enumerate(reg):
                    if i in kept:
                        continue
                    start = k - k % run
                    wit = [p0] + [j for j in reg[start:k] if j in kept]
                    assert any(_in_closed_triangle(pts[i], A, pts[w], B) for w in wit), (t, bs, i)


def test_second_round_reverse_golden_trace():
    """The mirrored second round on the hand-made points of Section 2.2.3's
    trace (tests/golden/second_round_reverse_trace.json, derived by hand)."""
    with open(os.path.join(GOLDEN, "second_round_reverse_trace.json")) as f:
        g = json.load(f)
    names, P, perm = g["names"], g["points"], g["index_permutation"]
    pts = np.zeros((len(P), 2), np.int32)
    for k, j in enumerate(perm):
        pts[j] = P[k]
    name_of = {perm[k]: names[k] for k in range(len(names))}
    idx_of = {v: k for k, v in name_of.items()}
    st = oracle.gscan_stages(pts, reverse=True)
    assert [name_of[i] for i in st["lower_fwd"]] == g["forward_lower_kept"]
    assert [name_of[i] for i in st["upper_fwd"]] == g["forward_upper_kept"]
    assert [name_of[i] for i in st["lower"]] == g["expected_lower_reverse"]
    assert [name_of[i] for i in st["upper"]] == g["expected_upper_reverse"]
    assert [name_of[i] for i in st["hull"]] == g["expected_hull_ccw"]
    lo = oracle.second_round_reverse(pts, idx_of["P0"], [idx_of[q] for q in g["forward_lower_kept"]], idx_of["Pl"], +1)
    assert [name_of[i] for i in lo] == g["expected_lower_reverse"]


def test_second_round_reverse_is_safe_with_witnesses():
    """The mirrored second round keeps a subset of the forward survivors that
    still holds every strict hull vertex, and every point it removes lies in
    the closed triangle (P_0, P_temp, P_l), P_temp being the nearest kept
    point after it in sorted order (or P_l)."""
    rng = np.random.default_rng(31)
    for t in range(200):
        n = int(rng.integers(3, 60))
        pts = rand_tiny(rng, n, int(rng.choice([3, 8, 1000, 1 << 29])))
        srt = oracle.sort_survivors(pts, np.arange(n))
        lo, up, lpos = oracle.second_round(pts, srt)
        if lpos < 0:
            continue
        p0, pl = int(srt[0]), int(srt[lpos])
        hv = set(brute_hull(pts))
        for region, sign in ((lo, +1), (up, -1)):
            rev = oracle.second_round_reverse(pts, p0, region, pl, sign)
            assert set(rev.tolist()) <= set(region.tolist())
            pos = {int(j): k for k, j in enumerate(region)}
            assert [pos[int(j)] for j in rev] == sorted(pos[int(j)] for j in rev)
            kept = set(rev.tolist())
            for k, j in enumerate(region):
                j = int(j)
                if j in kept:
                    continue
                assert j not in hv, (t, j)
                later = [int(q) for q in region[k + 1:] if int(q) in kept]
                T = later[0] if later else pl
                assert _in_closed_triangle(pts[j], pts[p0], pts[T], pts[pl]), (t, j)


def test_second_round_reverse_keeps_convex_chains():
    """On points in strictly convex position every forward survivor is a hull
    vertex, and the mirrored pass keeps them all."""
    par = W.parabola_lattice(1 << 10)
    rng = np.random.default_rng(32)
    for pts in (par, par[rng.permutation(len(par))]):
        st = oracle.gscan_stages(pts, reverse=True)
        assert st["lower"].tolist() == st["lower_fwd"].tolist()
        assert st["upper"].tolist() == st["upper_fwd"].tolist()
        assert len(st["lower"]) == len(pts) - 2


def test_method_with_reverse_equals_definition():
    """Both second rounds, then the stack scan, give exactly the hull."""
    rng = np.random.default_rng(33)
    for t in range(300):
        n = int(rng.integers(0, 200))
        pts = rand_tiny(rng, n, int(rng.choice([1, 3, 20, 1 << 29])))
        assert oracle.gscan_stages(pts, reverse=True)["hull"].tolist() == oracle.hull(pts).tolist()
    for f in (lambda: W.uniform_square(200000, 1 << 29, 41), lambda: W.uniform_disk(200000, 2.0 ** 29, 42),
              lambda: W.near_circle(100000, 2.0 ** 20, 43), lambda: W.gaussian_clusters(100000, 44)):
        pts = f()
        assert oracle.gscan_stages(pts, reverse=True)["hull"].tolist() == oracle.hull(pts).tolist()


def test_method_equals_definition():
    """Sections 2.2.2 and 5.2: the two filtering rounds followed by the stack
    scan give exactly the hull of all points."""
    rng = np.random.default_rng(12)
    for t in range(300):
        n = int(rng.integers(0, 200))
        pts = rand_tiny(rng, n, int(rng.choice([1, 3, 20, 1 << 29])))
        assert oracle.gscan_stages(pts)["hull"].tolist() == oracle.hull(pts).tolist()
    for f in (lambda: W.uniform_square(200000, 1 << 29, 21), lambda: W.uniform_disk(200000, 2.0 ** 29, 22),
              lambda: W.near_circle(100000, 2.0 ** 20, 23), lambda: W.gaussian_clusters(100000, 24)):
        pts = f()
        assert oracle.gscan_stages(pts)["hull"].tolist() == oracle.hull(pts).tolist()


# ---------------------------------------------------------------- chain

def test_chain_matches_brute_force_lower_upper():
    rng = np.random.default_rng(13)
    for t in range(200):
        n = int(rng.integers(2, 40))
        pts = rand_tiny(rng, n, int(rng.choice([3, 50])))
        u = np.unique(pts, axis=0)              # lexicographically sorted, distinct
        if len(u) < 2:
            continue
        lo = u[oracle.chain(u, +1)]
        up = u[oracle.chain(u, -1)]
        bh = brute_hull(u)
        hv = u[bh].tolist()
        # lower chain = CCW hull from the min up to the max; upper = the rest
        imax = hv.index(u[-1].tolist())
        assert lo.tolist() == hv[: imax + 1]
        assert up.tolist() == [hv[0]] + hv[imax + 1:][::-1] + [hv[imax]]
