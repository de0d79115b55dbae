"""CPU oracle for the gScan hot path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The library's product path never
does: it shares no code with the CUDA kernels and the two never import each
other.

Every function follows a passage of Mei, "gScan: Accelerating Graham Scan on
the GPU" (arXiv 1508.05931), cited in its docstring, and is pinned by the
``-m "not gpu"`` tests in ``tests/test_oracle_pins.py`` to brute force,
closed forms and invariants.  Pinning status per function:

* ``hull``            pinned (O(n^3) brute force, closed forms, invariants)
* ``extremes``        pinned (lexsort library routine, brute force)
* ``quad_filter``     pinned (exact rational point-in-polygon, statistics)
* ``sort_survivors``  pinned (numpy lexsort; a library primitive)
* ``second_round``    pinned (triangle witnesses, hull superset, Section
                      2.2.3's worked P_temp trace)
* ``second_round_chunked`` pinned (one run = the exact second round, runs of
                      one point keep the whole region, a superset of the exact
                      survivors holding every hull vertex, triangle witnesses)
* ``second_round_reverse`` pinned (triangle witnesses, hull superset, subset of
                      the forward survivors, convex chains kept whole, a
                      hand-derived trace)
* ``chain``           pinned (brute force on sorted input)
* ``angular_sort``, ``angular_second_round``, ``graham``, ``angular_stages``
                      (the paper's own angular ordering) pinned (exact
                      rational slopes and fp64 atan2 for the order; the hull
                      by definition and brute force; hull superset; a
                      hand-derived trace of both walks)
* the learned-proposal MLP (``oracle.mlp``) is pinned by finite differences
  and a closed-form tiny network.

The C part (``hull_oracle.c``) is compiled with plain gcc, no vector
intrinsics, by ``build()``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hull_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle_hull.so")
_lib = None

COORD_LIMIT = 1 << 29


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc into oracle/_build/liboracle_hull.so."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    P = ctypes.c_void_p
    I64 = ctypes.c_int64
    lib.oracle_range_ok.argtypes = [P, I64]
    lib.oracle_range_ok.restype = ctypes.c_int
    lib.oracle_chain.argtypes = [P, I64, ctypes.c_int, P]
    lib.oracle_chain.restype = I64
    lib.oracle_hull.argtypes = [P, I64, P]
    lib.oracle_hull.restype = I64
    lib.oracle_extremes.argtypes = [P, I64, P]
    lib.oracle_extremes.restype = ctypes.c_int
    lib.oracle_quad.argtypes = [P, I64, P]
    lib.oracle_quad.restype = ctypes.c_int
    lib.oracle_quad_filter.argtypes = [P, I64, P]
    lib.oracle_quad_filter.restype = I64
    lib.oracle_second_round.argtypes = [P, I64, P, P, P, P, P]
    lib.oracle_second_round.restype = ctypes.c_int
    lib.oracle_second_round_chunked.argtypes = [P, I64, I64, P, P, P, P, P]
    lib.oracle_second_round_chunked.restype = ctypes.c_int
    lib.oracle_second_round_reverse.argtypes = [P, I64, ctypes.c_int, P, P]
    lib.oracle_second_round_reverse.restype = ctypes.c_int
    lib.oracle_sort_xyi.argtypes = [P, I64]
    lib.oracle_sort_xyi.restype = None
    lib.oracle_angular_sort.argtypes = [P, I64, P]
    lib.oracle_angular_sort.restype = None
    lib.oracle_angular_second_round.argtypes = [P, I64, P]
    lib.oracle_angular_second_round.restype = I64
    lib.oracle_graham.argtypes = [P, I64, P]
    lib.oracle_graham.restype = I64
    _lib = lib
    return lib


def _pts(xy) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(xy, dtype=np.int32).reshape(-1, 2))
    return a


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def range_ok(xy) -> bool:
    a = _pts(xy)
    return bool(_load().oracle_range_ok(_ptr(a), a.shape[0]))


def hull(xy) -> np.ndarray:
    """Convex hull by definition (Section 1), Andrew's monotone chain over all
    points; CCW input indices from the lexicographic minimum, collinear
    boundary points excluded, smallest index among duplicates.
    Raises ValueError for coordinates beyond +-2^29."""
    a = _pts(xy)
    n = a.shape[0]
    out = np.empty(max(n, 1), dtype=np.int32)
    h = _load().oracle_hull(_ptr(a), n, _ptr(out))
    if h == -1:
        raise ValueError("coordinate out of range")
    if h < 0:
        raise MemoryError("oracle allocation failed")
    return out[:h].copy()


def extremes(xy) -> np.ndarray:
    """Section 2.1 step 1: [P_minx, P_maxx, P_miny, P_maxy] indices with
    lexicographic ties and the smallest index."""
    a = _pts(xy)
    ext = np.full(4, -1, dtype=np.int32)
    _load().oracle_extremes(_ptr(a), a.shape[0], _ptr(ext))
    return ext


def quad(xy) -> np.ndarray:
    """Distinct corners (k, 2) of the first-round polygon, CCW from P_minx."""
    a = _pts(xy)
    poly = np.zeros(8, dtype=np.int32)
    k = _load().oracle_quad(_ptr(a), a.shape[0], _ptr(poly))
    return poly[: 2 * k].reshape(k, 2).copy()


def quad_filter(xy) -> np.ndarray:
    """Section 3.1: ascending indices of points NOT strictly inside the quad."""
    a = _pts(xy)
    keep = np.empty(max(a.shape[0], 1), dtype=np.int32)
    s = _load().oracle_quad_filter(_ptr(a), a.shape[0], _ptr(keep))
    return keep[:s].copy()


def sort_survivors(xy, idx) -> np.ndarray:
    """Section 2.1 step 4, with the lexicographic key: the survivors' indices
    ordered by (x, y, idx) -- a stable sort of index-ordered survivors."""
    a = _pts(xy)
    idx = np.asarray(idx, dtype=np.int64)
    order = np.lexsort((idx, a[idx, 1], a[idx, 0]))
    return idx[order].astype(np.int32)


def second_round(xy, sorted_idx):
    """Figure 2 (Section 2.2) run sequentially over both regions of a list of
    input indices sorted by (x, y, idx).  Returns (lower_idx, upper_idx,
    l_pos) where the index lists are input indices in list order and l_pos
    is the list position of P_l (-1 if every point equals P_0)."""
    a = _pts(xy)
    sidx = np.asarray(sorted_idx, dtype=np.int64)
    m = sidx.shape[0]
    xyi = np.empty((m, 3), dtype=np.int32)
    xyi[:, :2] = a[sidx]
    xyi[:, 2] = sidx
    lo = np.empty(max(m, 1), dtype=np.int32)
    up = np.empty(max(m, 1), dtype=np.int32)
    nlo = ctypes.c_int64()
    nup = ctypes.c_int64()
    lp = ctypes.c_int64()
    _load().oracle_second_round(_ptr(xyi), m, _ptr(lo), ctypes.byref(nlo), _ptr(up),
                                ctypes.byref(nup), ctypes.byref(lp))
    lo_pos = lo[: nlo.value]
    up_pos = up[: nup.value]
    return (sidx[lo_pos].astype(np.int32), sidx[up_pos].astype(np.int32), int(lp.value))


def second_round_chunked(xy, sorted_idx, block_size: int = 1024):
    """Section 3.4: the second round with each region split into block_size
    runs of ceil(m / block_size) consecutive points (m = the region's
    points), Figure 2 run over every run on its own from P_temp = P_0.
    Returns (lower_idx, upper_idx, l_pos) like second_round."""
    a = _pts(xy)
    sidx = np.asarray(sorted_idx, dtype=np.int64)
    m = sidx.shape[0]
    xyi = np.empty((m, 3), dtype=np.int32)
    xyi[:, :2] = a[sidx]
    xyi[:, 2] = sidx
    lo = np.empty(max(m, 1), dtype=np.int32)
    up = np.empty(max(m, 1), dtype=np.int32)
    nlo, nup, lp = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    _load().oracle_second_round_chunked(_ptr(xyi), m, int(block_size), _ptr(lo), ctypes.byref(nlo), _ptr(up),
                                        ctypes.byref(nup), ctypes.byref(lp))
    return (sidx[lo[: nlo.value]].astype(np.int32), sidx[up[: nup.value]].astype(np.int32), int(lp.value))


def second_round_reverse(xy, p0, region, pl, sign: int) -> np.ndarray:
    """The second round mirrored over one region's forward survivors (the
    reverse pass of Figure 2, Section 2.2, applied to its own output): the
    list P_0 (input index p0), `region` (input indices in sorted order), P_l
    (index pl) is walked from P_l back toward P_0 with P_0 as the anchor; a
    point is kept when it lies strictly below (sign = +1, lower region) or
    above (sign = -1, upper) the line from the running P_temp (initially P_l)
    to P_0, and then becomes P_temp.  Returns the kept input indices in
    sorted order."""
    a = _pts(xy)
    seq = np.concatenate([[p0], np.asarray(region, dtype=np.int64), [pl]]).astype(np.int64)
    lst = np.ascontiguousarray(a[seq])
    keep = np.empty(max(len(seq), 1), dtype=np.int32)
    nk = ctypes.c_int64()
    _load().oracle_second_round_reverse(_ptr(lst), len(seq), int(sign), _ptr(keep), ctypes.byref(nk))
    return seq[keep[: nk.value]].astype(np.int32)


def chain(xy_seq, sign: int) -> np.ndarray:
    """Stack-based monotone chain (Section 2.1 step 8, Section 5.2) over a
    sequence of points given in lexicographic order; sign +1 = lower chain,
    -1 = upper chain walked left to right.  Returns kept positions."""
    a = _pts(xy_seq)
    m = a.shape[0]
    xyi = np.zeros((m, 3), dtype=np.int32)
    xyi[:, :2] = a
    out = np.empty(max(m, 1), dtype=np.int32)
    h = _load().oracle_chain(_ptr(xyi), m, int(sign), _ptr(out))
    return out[:h].copy()


def gscan_stages(xy, reverse: bool = False):
    """The method's stages in the paper's order (Section 2.1 steps 1-8),
    each computed by the functions above.  Returns a dict of intermediates
    and the final CCW hull built from the second-round survivors; with
    `reverse`, the mirrored second round also runs over both regions
    (keys lower_fwd / upper_fwd keep the forward survivors) and the hull is
    built from its survivors."""
    a = _pts(xy)
    n = a.shape[0]
    out = {"n": n}
    if n == 0:
        out.update(ext=np.full(4, -1, np.int32), keep=np.zeros(0, np.int32),
                   sorted=np.zeros(0, np.int32), lower=np.zeros(0, np.int32),
                   upper=np.zeros(0, np.int32), hull=np.zeros(0, np.int32))
        return out
    out["ext"] = extremes(a)
    keep = quad_filter(a)
    out["keep"] = keep
    srt = sort_survivors(a, keep)
    out["sorted"] = srt
    lo, up, lpos = second_round(a, srt)
    out["lower"], out["upper"] = lo, up
    if lpos < 0:
        out["hull"] = srt[:1].copy()
        return out
    p0, pl = int(srt[0]), int(srt[lpos])
    if reverse:
        out["lower_fwd"], out["upper_fwd"] = lo, up
        lo = second_round_reverse(a, p0, lo, pl, +1)
        up = second_round_reverse(a, p0, up, pl, -1)
        out["lower"], out["upper"] = lo, up
    lo_seq = np.concatenate([[p0], lo, [pl]]).astype(np.int64)
    up_seq = np.concatenate([[p0], up, [pl]]).astype(np.int64)
    lc = lo_seq[chain(a[lo_seq], +1)]
    uc = up_seq[chain(a[up_seq], -1)]
    out["hull"] = np.concatenate([lc, uc[1:-1][::-1]]).astype(np.int32)
    return out


# ------------------------------------------------------- the angular variant

def _triples(a: np.ndarray, idx) -> np.ndarray:
    idx = np.asarray(idx, dtype=np.int64)
    t = np.empty((idx.shape[0], 3), dtype=np.int32)
    t[:, :2] = a[idx]
    t[:, 2] = idx
    return t


def angular_sort(xy, idx, anchor: int) -> np.ndarray:
    """Section 2.1 steps 3-4 (Sections 3.2-3.3): the indices `idx` ordered by
    their angle about the point xy[anchor], ascending; points equal to the
    anchor (the anchor included) are left out.  The anchor must be the
    lowest point, leftmost among the lowest, so that every angle is in
    [0, pi).  Equal angles: nearer first, then the smaller index."""
    a = _pts(xy)
    idx = np.asarray(idx, dtype=np.int64)
    idx = idx[(a[idx, 0] != a[anchor, 0]) | (a[idx, 1] != a[anchor, 1])]
    t = _triples(a, idx)
    at = _triples(a, [anchor])
    _load().oracle_angular_sort(_ptr(t), t.shape[0], _ptr(at))
    return t[:, 2].copy()


def angular_second_round(xy, order):
    """Sections 2.1 steps 5-7 and 2.2, Figure 2 as printed, over `order` =
    [anchor, its points in angular order]: P_l is the point farthest from
    the anchor, the right region (positions 1 .. l - 1) is walked forward
    from P_0, the left region (l + 1 .. m - 2) backward from P_{m-1}.
    Returns (keep, l): keep[i] tells whether position i survives (P_0, P_l
    and P_{m-1} always do); l = -1 when the list holds the anchor alone."""
    a = _pts(xy)
    t = _triples(a, order)
    keep = np.zeros(max(t.shape[0], 1), dtype=np.uint8)
    l = _load().oracle_angular_second_round(_ptr(t), t.shape[0], _ptr(keep))
    return keep[: t.shape[0]].astype(bool), int(l)


def graham(xy, seq) -> np.ndarray:
    """Section 2.1 step 8 read as Graham's scan over `seq` = [anchor, points
    in angular order]: returns the hull as input indices, counter-clockwise
    from the anchor, strict vertices only."""
    a = _pts(xy)
    t = _triples(a, seq)
    out = np.empty(max(t.shape[0], 1), dtype=np.int32)
    h = _load().oracle_graham(_ptr(t), t.shape[0], _ptr(out))
    return t[out[:h], 2].astype(np.int32)


def angular_stages(xy):
    """The method with the paper's angular ordering, in its order (Section
    2.1 steps 1-8): extremes, the quadrilateral filter, the angular sort
    about P_miny, P_longest and the two walks of Figure 2, Graham's scan.
    Returns a dict of intermediates: anchor, keep (first-round survivors),
    order ([anchor] + angular order), l_pos, kept (the second round's
    survivors of `order`, a boolean mask), survivors (their indices, in
    order) and hull (counter-clockwise from the anchor)."""
    a = _pts(xy)
    out = {"n": a.shape[0]}
    if a.shape[0] == 0:
        z = np.zeros(0, np.int32)
        out.update(anchor=-1, keep=z, order=z, l_pos=-1, kept=np.zeros(0, bool), survivors=z, hull=z)
        return out
    anchor = int(extremes(a)[2])
    keep = quad_filter(a)
    order = np.concatenate([[anchor], angular_sort(a, keep, anchor)]).astype(np.int32)
    kept, l = angular_second_round(a, order)
    surv = order[kept]
    out.update(anchor=anchor, keep=keep, order=order, l_pos=l, kept=kept, survivors=surv,
               hull=graham(a, surv))
    return out

