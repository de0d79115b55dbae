/*
 * CPU oracle for the gScan hot path (Mei, "gScan: Accelerating Graham Scan
 * on the GPU", arXiv 1508.05931).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library's product path links,
 * loads or calls this file; only the tests, the smoke check and the CPU
 * baseline leg of the benchmark do.  It shares no code, header or table with
 * the CUDA path.  Plain, sequential, int64 arithmetic throughout.
 *
 * Conventions (the readings this oracle takes where the paper is silent):
 *   - a point is (x, y) with |x|, |y| <= 2^29; cross products are exact int64;
 *   - orient(a, b, c) = (b - a) x (c - a); "left of a->b" means > 0;
 *   - the hull is the set of strict vertices (collinear boundary points are
 *     excluded), reported counter-clockwise starting at the lexicographically
 *     smallest (x, y), with the smallest input index among equal points.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_COORD_LIMIT (1 << 29)

typedef struct {
    int32_t x, y, idx;
} opt_t;

static int64_t orient(const opt_t *a, const opt_t *b, const opt_t *c)
{
    int64_t bx = (int64_t)b->x - a->x, by = (int64_t)b->y - a->y;
    int64_t cx = (int64_t)c->x - a->x, cy = (int64_t)c->y - a->y;
    return bx * cy - by * cx;
}

static int cmp_xyi(const void *pa, const void *pb)
{
    const opt_t *a = (const opt_t *)pa, *b = (const opt_t *)pb;
    if (a->x != b->x) return a->x < b->x ? -1 : 1;
    if (a->y != b->y) return a->y < b->y ? -1 : 1;
    if (a->idx != b->idx) return a->idx < b->idx ? -1 : 1;
    return 0;
}

static int same_xy(const opt_t *a, const opt_t *b) { return a->x == b->x && a->y == b->y; }

/* 1 if every coordinate is within +-2^29, else 0. */
int oracle_range_ok(const int32_t *xy, int64_t n)
{
    for (int64_t i = 0; i < 2 * n; ++i)
        if (xy[i] > ORACLE_COORD_LIMIT || xy[i] < -ORACLE_COORD_LIMIT) return 0;
    return 1;
}

/*
 * Monotone chain over a sequence that is already in lexicographic (x, y)
 * order (Andrew's form of Graham's scan, the stack-based finalisation of
 * Section 2.1 step 8 and Section 5.2): for each point in the given order,
 * pop while the last two kept points and the new one do not make a strict
 * turn of the requested sign, then push.  sign = +1 builds the lower chain
 * (left turns), sign = -1 the upper chain walked left to right.
 * Writes the kept positions (0-based into pts) to out; returns their count.
 */
int64_t oracle_chain(const int32_t *xyi, int64_t m, int sign, int32_t *out)
{
    const opt_t *p = (const opt_t *)xyi;
    int64_t h = 0;
    for (int64_t i = 0; i < m; ++i) {
        while (h >= 2) {
            int64_t o = orient(&p[out[h - 2]], &p[out[h - 1]], &p[i]);
            if ((sign > 0 && o <= 0) || (sign < 0 && o >= 0)) --h;
            else break;
        }
        out[h++] = (int32_t)i;
    }
    return h;
}

/*
 * The convex hull by its plain definition (Section 1: the smallest polygon
 * that contains every point), computed by Andrew's monotone chain over ALL
 * points: sort (x, y, idx), drop repeated (x, y) keeping the smallest idx,
 * lower chain ascending, upper chain descending, both popping on
 * orientation <= 0.  Output: CCW input indices from the lexicographic
 * minimum.  Returns h, or -1 if a coordinate is out of range, or -2 on
 * allocation failure.  out needs room for min(n, 2 * n) entries (n is
 * enough).
 */
int64_t oracle_hull(const int32_t *xy, int64_t n, int32_t *out)
{
    if (n <= 0) return 0;
    if (!oracle_range_ok(xy, n)) return -1;
    opt_t *p = (opt_t *)malloc((size_t)n * sizeof(opt_t));
    opt_t **st = (opt_t **)malloc((size_t)(2 * n + 2) * sizeof(opt_t *));
    if (!p || !st) { free(p); free(st); return -2; }
    for (int64_t i = 0; i < n; ++i) { p[i].x = xy[2 * i]; p[i].y = xy[2 * i + 1]; p[i].idx = (int32_t)i; }
    qsort(p, (size_t)n, sizeof(opt_t), cmp_xyi);
    int64_t m = 0;
    for (int64_t i = 0; i < n; ++i)
        if (m == 0 || !same_xy(&p[m - 1], &p[i])) p[m++] = p[i];
    if (m == 1) { out[0] = p[0].idx; free(p); free(st); return 1; }
    int64_t k = 0;
    for (int64_t i = 0; i < m; ++i) {                 /* lower chain */
        while (k >= 2 && orient(st[k - 2], st[k - 1], &p[i]) <= 0) --k;
        st[k++] = &p[i];
    }
    int64_t lower = k;
    for (int64_t i = m - 2; i >= 0; --i) {            /* upper chain */
        while (k > lower && orient(st[k - 2], st[k - 1], &p[i]) <= 0) --k;
        st[k++] = &p[i];
    }
    int64_t h = k - 1;                                /* last equals first */
    for (int64_t i = 0; i < h; ++i) out[i] = st[i]->idx;
    free(p); free(st);
    return h;
}

/*
 * Section 2.1 step 1 / Section 3.1: the four extreme points.  Ties are
 * broken lexicographically and then by the smallest index:
 *   ext[0] = P_minx = argmin (x, y, idx)     ext[1] = P_maxx = argmax (x, y), min idx
 *   ext[2] = P_miny = argmin (y, x, idx)     ext[3] = P_maxy = argmax (y, x), min idx
 * Returns 0 and leaves ext untouched when n <= 0.
 */
int oracle_extremes(const int32_t *xy, int64_t n, int32_t *ext)
{
    if (n <= 0) return 0;
    int64_t a = 0, b = 0, c = 0, d = 0;
    for (int64_t i = 1; i < n; ++i) {
        int32_t x = xy[2 * i], y = xy[2 * i + 1];
        int32_t ax = xy[2 * a], ay = xy[2 * a + 1];
        int32_t bx = xy[2 * b], by = xy[2 * b + 1];
        int32_t cx = xy[2 * c], cy = xy[2 * c + 1];
        int32_t dx = xy[2 * d], dy = xy[2 * d + 1];
        if (x < ax || (x == ax && y < ay)) a = i;
        if (x > bx || (x == bx && y > by)) b = i;
        if (y < cy || (y == cy && x < cx)) c = i;
        if (y > dy || (y == dy && x > dx)) d = i;
    }
    ext[0] = (int32_t)a; ext[1] = (int32_t)b; ext[2] = (int32_t)c; ext[3] = (int32_t)d;
    return 1;
}

/*
 * The first-round filter polygon (Section 2.1 step 2, Section 3.1): corners
 * in the cyclic order P_minx, P_miny, P_maxx, P_maxy (counter-clockwise
 * along the hull), with cyclically repeated points removed.  Writes up to 4
 * (x, y) pairs to poly; returns the number of distinct corners.
 */
int oracle_quad(const int32_t *xy, int64_t n, int32_t *poly)
{
    int32_t ext[4];
    if (!oracle_extremes(xy, n, ext)) return 0;
    const int order[4] = {0, 2, 1, 3};
    int32_t cx[4], cy[4];
    int k = 0;
    for (int j = 0; j < 4; ++j) {
        int32_t x = xy[2 * (int64_t)ext[order[j]]], y = xy[2 * (int64_t)ext[order[j]] + 1];
        if (k > 0 && cx[k - 1] == x && cy[k - 1] == y) continue;
        cx[k] = x; cy[k] = y; ++k;
    }
    while (k > 1 && cx[k - 1] == cx[0] && cy[k - 1] == cy[0]) --k;
    for (int j = 0; j < k; ++j) { poly[2 * j] = cx[j]; poly[2 * j + 1] = cy[j]; }
    return k;
}

/*
 * Section 3.1: a point is discarded when it lies strictly inside the
 * quadrilateral, i.e. strictly left of every counter-clockwise edge; with
 * fewer than three distinct corners nothing is discarded.  Writes the kept
 * input indices in ascending order to keep; returns their count.
 */
int64_t oracle_quad_filter(const int32_t *xy, int64_t n, int32_t *keep)
{
    int32_t poly[8];
    int k = oracle_quad(xy, n, poly);
    int64_t s = 0;
    for (int64_t i = 0; i < n; ++i) {
        opt_t p = {xy[2 * i], xy[2 * i + 1], 0};
        int inside = (k >= 3);
        for (int j = 0; j < k && inside; ++j) {
            opt_t a = {poly[2 * j], poly[2 * j + 1], 0};
            opt_t b = {poly[2 * ((j + 1) % k)], poly[2 * ((j + 1) % k) + 1], 0};
            if (orient(&a, &b, &p) <= 0) inside = 0;
        }
        if (!inside) keep[s++] = (int32_t)i;
    }
    return s;
}

/*
 * Sections 2.1 steps 5-7 and 2.2, Figure 2, run sequentially over a list
 * already sorted in lexicographic (x, y, idx) order (triples x, y, idx).
 * P_0 is the first point (P_minx); P_l ("longest", the end of both walks) is
 * the first point of the last run of equal (x, y) (P_maxx).  Each point is
 * assigned to the region strictly right of the directed line P_0 -> P_l
 * (lower) or strictly left of it (upper); points on the line are dropped.
 * Both regions are walked from P_0 towards P_l with a running P_temp that
 * starts at P_0: a lower point is interior when it lies left of or on the
 * line P_temp -> P_l, an upper point when it lies right of or on it;
 * otherwise it is kept and becomes P_temp.
 * Writes the kept positions (0-based into the list) of each region in list
 * order.  Returns 0 on success; counts in *n_lo, *n_up; *l_pos = position
 * of P_l (or -1 when every point coincides with P_0).
 */
int oracle_second_round(const int32_t *xyi, int64_t m, int32_t *lo, int64_t *n_lo,
                        int32_t *up, int64_t *n_up, int64_t *l_pos)
{
    const opt_t *p = (const opt_t *)xyi;
    *n_lo = 0; *n_up = 0; *l_pos = -1;
    if (m <= 0) return 0;
    int64_t l = m - 1;
    while (l > 0 && same_xy(&p[l - 1], &p[m - 1])) --l;
    if (same_xy(&p[0], &p[l])) return 0;
    *l_pos = l;
    const opt_t *t_lo = &p[0], *t_up = &p[0];
    for (int64_t i = 1; i < m; ++i) {
        int64_t side = orient(&p[0], &p[l], &p[i]);
        if (side < 0) {
            if (orient(t_lo, &p[l], &p[i]) < 0) { lo[(*n_lo)++] = (int32_t)i; t_lo = &p[i]; }
        } else if (side > 0) {
            if (orient(t_up, &p[l], &p[i]) > 0) { up[(*n_up)++] = (int32_t)i; t_up = &p[i]; }
        }
    }
    return 0;
}

/* Section 3.4's chunked second round: the region's points (in sorted
 * order) are split into `bs` runs of ceil(m_region / bs) consecutive points,
 * and Figure 2 runs over every run on its own, P_temp starting at P_0.
 * Same inputs and outputs as oracle_second_round. */
int oracle_second_round_chunked(const int32_t *xyi, int64_t m, int64_t bs, int32_t *lo, int64_t *n_lo,
                                int32_t *up, int64_t *n_up, int64_t *l_pos)
{
    const opt_t *p = (const opt_t *)xyi;
    *n_lo = 0; *n_up = 0; *l_pos = -1;
    if (m <= 0 || bs < 1) return 0;
    int64_t l = m - 1;
    while (l > 0 && same_xy(&p[l - 1], &p[m - 1])) --l;
    if (same_xy(&p[0], &p[l])) return 0;
    *l_pos = l;
    for (int r = 0; r < 2; ++r) {
        /* the region's positions, in order */
        int64_t cnt = 0;
        for (int64_t i = 1; i < m; ++i) {
            const int64_t side = orient(&p[0], &p[l], &p[i]);
            if ((r == 0 && side < 0) || (r == 1 && side > 0)) ++cnt;
        }
        const int64_t run = (cnt + bs - 1) / bs;
        int64_t k = 0;
        const opt_t *t = &p[0];
        int32_t *out = r == 0 ? lo : up;
        int64_t *nout = r == 0 ? n_lo : n_up;
        for (int64_t i = 1; i < m; ++i) {
            const int64_t side = orient(&p[0], &p[l], &p[i]);
            if (!((r == 0 && side < 0) || (r == 1 && side > 0))) continue;
            if (run > 0 && k % run == 0) t = &p[0];      /* a new run starts */
            const int64_t o = orient(t, &p[l], &p[i]);
            if ((r == 0 && o < 0) || (r == 1 && o > 0)) { out[(*nout)++] = (int32_t)i; t = &p[i]; }
            ++k;
        }
    }
    return 0;
}

/* The second round mirrored (the reverse pass of Figure 2 applied to its
 * own survivors): p[0..m) is a region list -- P_0, the region's survivors
 * of the forward pass in sorted order, P_l.  The walk goes from P_l back
 * toward P_0 with P_0 as the anchor and a running P_temp that starts at
 * P_l; p[i] is kept when orient(P_temp, P_0, p[i]) is strictly positive
 * (lower region, sgn = +1: strictly below the line from P_temp to P_0) or
 * strictly negative (upper region, sgn = -1), and then becomes P_temp.  It
 * is Figure 2 on the point set reflected through x -> -x, where P_l is the
 * first point and P_0 the last (a reflection flips orient's sign).
 * keep[] receives the kept positions among 1 .. m - 2 in ascending order. */
int oracle_second_round_reverse(const int32_t *xy, int64_t m, int sgn, int32_t *keep, int64_t *n_keep)
{
    *n_keep = 0;
    if (m < 3) return 0;
    const int32_t *p0 = &xy[0];
    int64_t t = m - 1;
    int64_t k = 0;
    for (int64_t i = m - 2; i >= 1; --i) {
        const int32_t *pt = &xy[2 * t], *pi = &xy[2 * i];
        const int64_t o = ((int64_t)p0[0] - pt[0]) * ((int64_t)pi[1] - pt[1]) -
                          ((int64_t)p0[1] - pt[1]) * ((int64_t)pi[0] - pt[0]);
        if ((sgn > 0 && o > 0) || (sgn < 0 && o < 0)) {
            keep[k++] = (int32_t)i;
            t = i;
        }
    }
    for (int64_t a = 0, b = k - 1; a < b; ++a, --b) {
        const int32_t v = keep[a]; keep[a] = keep[b]; keep[b] = v;
    }
    *n_keep = k;
    return 0;
}

/* Stable sort of (x, y, idx) triples by (x, y, idx); used for the sort stage. */
void oracle_sort_xyi(int32_t *xyi, int64_t m)
{
    qsort(xyi, (size_t)m, sizeof(opt_t), cmp_xyi);
}

/*
 * The paper's own ordering (Section 2.1 steps 3-4, Sections 3.2-3.3): the
 * points sorted by their angle about an anchor, ascending.  Readings (the
 * paper names neither the anchor nor a tie rule): the anchor is P_miny =
 * argmin (y, x, idx), the pivot of Graham's scan, so every other point not
 * equal to it lies in dy > 0 or (dy == 0, dx > 0) and its angle about the
 * anchor is in [0, pi); inside that half-plane angle(a) < angle(b) exactly
 * when orient(anchor, a, b) > 0, so the order is decided by an exact int64
 * cross product, never by a rounded angle.  Equal angles are ordered by the
 * squared distance to the anchor (the distance of Section 3.2), then by
 * index.  The triples p[0 .. m) must not coincide with the anchor.
 */
static opt_t g_anchor;

static int cmp_angle(const void *pa, const void *pb)
{
    const opt_t *a = (const opt_t *)pa, *b = (const opt_t *)pb;
    const int64_t o = orient(&g_anchor, a, b);
    if (o != 0) return o > 0 ? -1 : 1;
    const int64_t ax = (int64_t)a->x - g_anchor.x, ay = (int64_t)a->y - g_anchor.y;
    const int64_t bx = (int64_t)b->x - g_anchor.x, by = (int64_t)b->y - g_anchor.y;
    const int64_t da = ax * ax + ay * ay, db = bx * bx + by * by;
    if (da != db) return da < db ? -1 : 1;
    if (a->idx != b->idx) return a->idx < b->idx ? -1 : 1;
    return 0;
}

void oracle_angular_sort(int32_t *xyi, int64_t m, const int32_t *anchor_xyi)
{
    g_anchor.x = anchor_xyi[0];
    g_anchor.y = anchor_xyi[1];
    g_anchor.idx = anchor_xyi[2];
    qsort(xyi, (size_t)m, sizeof(opt_t), cmp_angle);
}

/*
 * Sections 2.1 steps 5-7 and 2.2, Figure 2 as printed, over a list in the
 * angular order above: p[0] is the anchor P_0, p[1 .. m) its points sorted
 * by angle.  P_l is the point farthest from P_0 (step 5; the first in list
 * order among equally far points).  The right region (step 6) is walked
 * forward: P_temp starts at P_0 and for i = 1 .. l - 1 the point P_i is
 * interior when it lies left of or on the directed line P_temp -> P_l,
 * otherwise it is kept and becomes P_temp.  The left region is walked
 * backward: P_temp starts at P_{m-1}, which stays, and for i = m - 2 down to
 * l + 1 the point P_i is interior when it lies right of or on the line
 * P_temp -> P_l, otherwise it is kept and becomes P_temp.  ("On the line"
 * counts as interior: such a point lies on the segment from P_temp to P_l,
 * so it is never a strict hull vertex.)  keep[i] receives 1 for P_0, P_l,
 * P_{m-1} and every kept point, else 0.  Returns l, or -1 when m < 2.
 */
int64_t oracle_angular_second_round(const int32_t *xyi, int64_t m, uint8_t *keep)
{
    const opt_t *p = (const opt_t *)xyi;
    if (m < 2) {
        if (m == 1) keep[0] = 1;
        return -1;
    }
    int64_t l = 1, best = -1;
    for (int64_t i = 1; i < m; ++i) {
        const int64_t dx = (int64_t)p[i].x - p[0].x, dy = (int64_t)p[i].y - p[0].y;
        const int64_t d = dx * dx + dy * dy;
        if (d > best) { best = d; l = i; }
    }
    for (int64_t i = 0; i < m; ++i) keep[i] = 0;
    keep[0] = 1;
    keep[l] = 1;
    keep[m - 1] = 1;
    const opt_t *t = &p[0];
    for (int64_t i = 1; i < l; ++i) {
        if (orient(t, &p[l], &p[i]) < 0) { keep[i] = 1; t = &p[i]; }
    }
    t = &p[m - 1];
    for (int64_t i = m - 2; i > l; --i) {
        if (orient(t, &p[l], &p[i]) > 0) { keep[i] = 1; t = &p[i]; }
    }
    return l;
}

/*
 * Section 2.1 step 8 read as Graham's scan over the survivors in angular
 * order (p[0] the anchor): for each point in order, a point equal to the top
 * of the stack is skipped (the first of equal points stays), then the stack
 * is popped while its last two points and the new one do not make a strict
 * left turn, then the point is pushed.  No closing pass is needed: points of
 * equal angle arrive nearer first, and a nearer point B on the ray of a
 * farther C makes a right turn A -> B -> C with any A of smaller angle (or a
 * straight one with A = P_0), so C pops it, on the last ray too.  Writes the
 * hull's positions (counter-clockwise from the anchor) to out; returns their
 * count.
 */
int64_t oracle_graham(const int32_t *xyi, int64_t m, int32_t *out)
{
    const opt_t *p = (const opt_t *)xyi;
    int64_t h = 0;
    for (int64_t i = 0; i < m; ++i) {
        if (h > 0 && same_xy(&p[out[h - 1]], &p[i])) continue;
        while (h >= 2 && orient(&p[out[h - 2]], &p[out[h - 1]], &p[i]) <= 0) --h;
        out[h++] = (int32_t)i;
    }
    return h;
}
