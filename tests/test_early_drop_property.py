"""The sort's early drop (Figure 2 applied per bin before the sort inside a
bin) checked on the CPU against the oracle's Figure 2.

The sorted survivors are cut into consecutive runs ("bins").  A region point
of a run is dropped when it is not strictly beyond the running P_temp that
Figure 2 holds when the walk reaches the run's first position (lower region:
left of or on P_temp -> P_l; upper: right of or on it).  That P_temp is read
from the oracle's own output -- the last kept point of the region before the
run, else P_0 -- so nothing of the walk is restated here.  The claims:

  * no dropped point is ever kept by Figure 2;
  * Figure 2 over the list without the dropped points keeps exactly the same
    points, in the same order;
  * with one point per run the drop test is Figure 2's test itself: the points
    not dropped are exactly the kept ones.

All CPU-only."""
import numpy as np
import pytest

import oracle
from paper_1508_05931_gb300 import workloads as W


def _orient(a, b, c):
    return (int(b[0]) - int(a[0])) * (int(c[1]) - int(a[1])) - (int(b[1]) - int(a[1])) * (int(c[0]) - int(a[0]))


def _sorted_survivors(xy):
    return oracle.sort_survivors(xy, oracle.quad_filter(xy))


def _dropped(xy, srt, lo, up, lpos, starts):
    """Positions (into srt) the early drop removes, for runs starting at
    `starts` (ascending, starts[0] == 0)."""
    p0, pl = xy[srt[0]], xy[srt[lpos]]
    pos_of = {int(v): i for i, v in enumerate(srt.tolist())}
    lo_pos = np.array([pos_of[int(v)] for v in lo], dtype=np.int64)
    up_pos = np.array([pos_of[int(v)] for v in up], dtype=np.int64)
    drop = []
    bounds = list(starts) + [len(srt)]
    for r in range(len(starts)):
        a, b = bounds[r], bounds[r + 1]
        k = np.searchsorted(lo_pos, a) - 1          # last lower point kept before the run
        t_lo = xy[srt[lo_pos[k]]] if k >= 0 else p0
        k = np.searchsorted(up_pos, a) - 1
        t_up = xy[srt[up_pos[k]]] if k >= 0 else p0
        for i in range(a, b):
            p = xy[srt[i]]
            side = _orient(p0, pl, p)
            if side < 0 and _orient(t_lo, pl, p) >= 0:      # lower region, within the prefix
                drop.append(i)
            elif side > 0 and _orient(t_up, pl, p) <= 0:    # upper region, within the prefix
                drop.append(i)
    return np.array(drop, dtype=np.int64)


def _inputs():
    yield "square", W.uniform_square(3000, 1 << 20, 11)
    yield "disk", W.uniform_disk(3000, float(1 << 20), 12)
    yield "near_circle", W.near_circle(2000, float(1 << 24), 13)
    yield "gaussian", W.gaussian(3000, float(1 << 18), 14)
    yield "grid", W.filled_grid(40, 30)
    rng = np.random.default_rng(15)
    yield "dups", rng.integers(-8, 9, size=(3000, 2)).astype(np.int32)      # heavy duplication
    yield "collinear", np.stack([np.arange(500), 2 * np.arange(500)], 1).astype(np.int32)


def _partitions(m, rng):
    yield "one run", np.array([0])
    yield "singletons", np.arange(m)
    for size in (2, 7, 64):
        yield f"runs of {size}", np.arange(0, m, size)
    cuts = np.unique(np.concatenate([[0], rng.integers(1, max(m, 2), size=max(1, m // 20))]))
    yield "random runs", cuts[cuts < m]


@pytest.mark.parametrize("name,xy", list(_inputs()), ids=[n for n, _ in _inputs()])
def test_early_drop_is_exact(name, xy):
    xy = np.ascontiguousarray(xy, dtype=np.int32)
    srt = _sorted_survivors(xy)
    lo, up, lpos = oracle.second_round(xy, srt)
    if lpos < 0:
        pytest.skip("every point coincides with P_0: no regions")
    kept = set(lo.tolist()) | set(up.tolist())
    rng = np.random.default_rng(len(srt))
    for label, starts in _partitions(len(srt), rng):
        drop = _dropped(xy, srt, lo, up, lpos, starts)
        dropped_idx = set(srt[drop].tolist())
        assert not (dropped_idx & kept), (name, label)
        rest = np.delete(srt, drop)
        lo2, up2, lpos2 = oracle.second_round(xy, rest)
        assert lo2.tolist() == lo.tolist() and up2.tolist() == up.tolist(), (name, label)
        assert rest[lpos2] == srt[lpos], (name, label)
        if label == "singletons":
            region = [i for i in range(len(srt)) if _orient(xy[srt[0]], xy[srt[lpos]], xy[srt[i]]) != 0]
            assert set(srt[region].tolist()) - dropped_idx == kept, name


def test_drop_removes_most_region_points_on_uniform_input():
    # the point of the drop: with runs of 256 of 10k survivors, most region
    # points are decided before any order inside their run is known (84 % here)
    xy = W.uniform_square(20000, 1 << 20, 21)
    srt = _sorted_survivors(xy)
    lo, up, lpos = oracle.second_round(xy, srt)
    drop = _dropped(xy, srt, lo, up, lpos, np.arange(0, len(srt), 256))
    assert len(drop) > 0.8 * len(srt)


@pytest.mark.parametrize("name,xy", [("square", W.uniform_square(6000, 1 << 20, 22)),
                                     ("disk", W.uniform_disk(6000, float(1 << 20), 23)),
                                     ("dups", np.random.default_rng(24).integers(-8, 9, size=(4000, 2)).astype(np.int32))],
                         ids=["square", "disk", "dups"])
def test_nested_drops_are_exact(name, xy):
    # a drop over coarse runs, then another over finer runs of what is left
    # (each against the prefix Figure 2 holds at its run's start): the kept
    # lists never change
    xy = np.ascontiguousarray(xy, dtype=np.int32)
    srt = _sorted_survivors(xy)
    lo, up, lpos = oracle.second_round(xy, srt)
    rest = np.delete(srt, _dropped(xy, srt, lo, up, lpos, np.arange(0, len(srt), 512)))
    lo1, up1, lpos1 = oracle.second_round(xy, rest)
    assert lo1.tolist() == lo.tolist() and up1.tolist() == up.tolist()
    rest2 = np.delete(rest, _dropped(xy, rest, lo1, up1, lpos1, np.arange(0, len(rest), 16)))
    lo2, up2, _ = oracle.second_round(xy, rest2)
    assert lo2.tolist() == lo.tolist() and up2.tolist() == up.tolist()
    assert len(rest2) <= len(rest) <= len(srt)
