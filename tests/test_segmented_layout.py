"""Index arithmetic of the batched segmented path (csrc/batched.cu:
k_seg_ext / k_seg_filter tile runs, k_batch mode 2's gather; csrc/api.cu:
the tile numbering), restated on the CPU: the instances' tiles are numbered
in order (tfirst), block b of G takes tiles [b T / G, (b + 1) T / G), split
into runs of one instance; a run covers points [lo, hi) of its instance
and leaves its survivors at [lo, lo + count) with the count at the run's
first tile (0 at its other tiles); the gather finds survivor i in the last
tile whose run start (exclusive prefix of the counts) is at most i.
Checked on random size lists and grid sizes: every point of every
instance in exactly one run, every run inside its instance and its tiles,
and every gathered position one stored survivor, each taken once."""
import numpy as np

TILE = 16384


def seg_of_tile(tfirst, t):
    lo, hi = 0, len(tfirst) - 2
    while lo < hi:
        mid = (lo + hi + 1) >> 1
        if tfirst[mid] <= t:
            lo = mid
        else:
            hi = mid - 1
    return lo


def runs(sizes, grid):
    tfirst = [0]
    for n in sizes:
        tfirst.append(tfirst[-1] + (n + TILE - 1) // TILE)
    T = tfirst[-1]
    out = []
    for b in range(min(grid, T)):
        G = min(grid, T)
        t, t1 = b * T // G, (b + 1) * T // G
        while t < t1:
            h = seg_of_tile(tfirst, t)
            tf, te = tfirst[h], min(t1, tfirst[h + 1])
            lo, hi = (t - tf) * TILE, min(sizes[h], (te - tf) * TILE)
            out.append((h, t, te, lo, hi))
            t = te
    return tfirst, out


def test_runs_cover_every_point_once():
    rng = np.random.default_rng(5)
    for trial in range(120):
        b = int(rng.integers(1, 40))
        sizes = [int(v) for v in rng.integers(1, 5 * TILE, size=b)]
        sizes[int(rng.integers(0, b))] = TILE * int(rng.integers(1, 4))      # whole tiles
        grid = int(rng.integers(1, 700))
        tfirst, rs = runs(sizes, grid)
        cover = [np.zeros(n, np.int32) for n in sizes]
        tiles_seen = np.zeros(tfirst[-1], np.int32)
        for h, t, te, lo, hi in rs:
            assert tfirst[h] <= t < te <= tfirst[h + 1]
            assert 0 <= lo < hi <= sizes[h]
            cover[h][lo:hi] += 1
            tiles_seen[t:te] += 1
        assert all((c == 1).all() for c in cover)
        assert (tiles_seen == 1).all()


def test_gather_takes_every_survivor_once():
    rng = np.random.default_rng(6)
    for trial in range(60):
        n = 2_097_144 if trial == 0 else int(rng.integers(1, 40 * TILE))
        sizes = [n]
        grid = int(rng.integers(1, 400))
        tfirst, rs = runs(sizes, grid)
        nt = tfirst[1]
        assert nt <= 128                   # fewer than the gather's block
        tcnt = np.zeros(nt, np.int64)
        stored = np.zeros(nt * TILE, bool)
        for h, t, te, lo, hi in rs:
            c = int(rng.integers(0, min(hi - lo, 3000) + 1)) if rng.random() < 0.8 else 0
            tcnt[t] = c                    # the run's first tile; its others keep 0
            stored[(t - tfirst[h]) * TILE:(t - tfirst[h]) * TILE + c] = True
        start = np.concatenate([[0], np.cumsum(tcnt)[:-1]])
        tot = int(tcnt.sum())
        i = np.arange(tot)
        tile = np.searchsorted(start, i, side="right") - 1      # the last start <= i
        # the kernel's binary search, on a few positions
        for q in rng.integers(0, max(tot, 1), size=min(tot, 200)):
            lo, hi = 0, nt - 1
            while lo < hi:
                mid = (lo + hi + 1) >> 1
                if start[mid] <= q:
                    lo = mid
                else:
                    hi = mid - 1
            assert lo == tile[q]
        off = i - start[tile]
        assert (off >= 0).all() and (off < tcnt[tile]).all()
        taken = tile * TILE + off
        assert len(np.unique(taken)) == tot
        assert stored[taken].all() and stored.sum() == tot
