"""The sample polygon's hull (csrc/k0_poly.cu, one lane per candidate): for
at most 32 points sorted by (x, y) and distinct, point i is a strict
lower-hull vertex when the most counter-clockwise direction p_i - p_j
(j < i) is strictly clockwise of the most clockwise direction p_k - p_i
(k > i) -- every left slope below every right slope -- and a strict
upper-hull vertex in the mirrored case; the first and the last point end
both chains.  The hull is the lower vertices in increasing index, then the
upper ones in decreasing index.  Restated here and checked against the
oracle's hull (the definition, pinned elsewhere) on random sets with
duplicates removed, collinear runs, vertical ties and coordinates at the
range limits."""
import numpy as np

import oracle


def cross(ax, ay, bx, by):
    return ax * by - ay * bx


def vertex_test_hull(pts):
    """pts: sorted, distinct (x, y) tuples; returns hull positions, CCW."""
    m = len(pts)
    lower, upper = [], []
    for i in range(m):
        px, py = pts[i]
        lj = uj = lk = uk = None
        for q in range(m):
            qx, qy = pts[q]
            if q < i:
                d = (px - qx, py - qy)
                if lj is None:
                    lj = uj = d
                if cross(*lj, *d) > 0:
                    lj = d
                if cross(*uj, *d) < 0:
                    uj = d
            elif q > i:
                e = (qx - px, qy - py)
                if lk is None:
                    lk = uk = e
                if cross(*lk, *e) < 0:
                    lk = e
                if cross(*uk, *e) > 0:
                    uk = e
        endp = i == 0 or i == m - 1
        if endp or cross(*lj, *lk) > 0:
            lower.append(i)
        if not endp and cross(*uj, *uk) < 0:
            upper.append(i)
    return lower + upper[::-1]


def _sets(rng, count):
    lim = (1 << 29) - 1
    for t in range(count):
        m = int(rng.integers(1, 33))
        kind = t % 5
        if kind == 0:
            p = rng.integers(-4, 5, size=(m, 2))
        elif kind == 1:
            p = rng.integers(-1000, 1001, size=(m, 2))
        elif kind == 2:                       # few distinct x: vertical ties
            p = np.stack([rng.integers(-2, 3, size=m), rng.integers(-50, 51, size=m)], axis=1)
        elif kind == 3:                       # collinear runs
            s = rng.integers(-20, 21, size=m)
            p = np.stack([3 * s, -2 * s + (rng.integers(0, 4, size=m) == 0)], axis=1)
        else:
            p = rng.integers(-lim, lim + 1, size=(m, 2))
        yield sorted(set(map(tuple, p.tolist())))


def test_vertex_test_is_the_hull():
    rng = np.random.default_rng(2024)
    for pts in _sets(rng, 6000):
        got = vertex_test_hull(pts)
        ref = oracle.hull(np.array(pts, dtype=np.int32).reshape(-1, 2)).tolist()
        assert got == ref, (pts, got, ref)


def test_planted_mistake_fails():
    """A non-strict lower test (left slopes at most the right ones) keeps
    collinear boundary points and must disagree with the hull."""
    def sloppy(pts):
        m = len(pts)
        out = []
        for i in range(m):
            if i == 0 or i == m - 1:
                out.append(i)
                continue
            px, py = pts[i]
            best_l = None
            for j in range(i):
                d = (px - pts[j][0], py - pts[j][1])
                if best_l is None or cross(*best_l, *d) > 0:
                    best_l = d
            best_r = None
            for k in range(i + 1, m):
                e = (pts[k][0] - px, pts[k][1] - py)
                if best_r is None or cross(*best_r, *e) < 0:
                    best_r = e
            if cross(*best_l, *best_r) >= 0:
                out.append(i)
        return out
    pts = [(0, 0), (1, 0), (2, 0), (2, 5)]
    lower_ref = [i for i in oracle.hull(np.array(pts, np.int32)).tolist() if i in (0, 1, 2, 3)]
    assert 1 not in lower_ref            # (1, 0) lies on the edge (0, 0) - (2, 0)
    assert 1 in sloppy(pts)
    assert 1 not in vertex_test_hull(pts)
