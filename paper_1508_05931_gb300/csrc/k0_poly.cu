// K0 of the single-read front: the sample polygon.
//
// Every kPolyStride-th point is projected on kPolyDirs directions u_j =
// (cos 2 pi j / D, sin 2 pi j / D) in float.  The sample's extreme point in
// each direction (largest projection, ties to the smallest sample index) is
// an input point, so the convex hull of those points is a polygon spanned by
// input points: a point strictly inside it is strictly inside the hull of the
// input and is no vertex of it (the argument of Section 2.2.2 for any filter
// polygon whose corners are input points).  The float projections only
// choose the corners; the polygon and the table built from it are exact.
//
// The last block builds the polygon (the strict convex hull of at most
// kPolyDirs points, counter-clockwise from the lexicographic minimum, one
// lane per point) and, for K1, a table over its x range (xl, xr) cut into slabs of
// 2^sh columns: for slab s an integer interval (ylo, yhi) with ylo at or
// above the lower chain and yhi at or below the upper chain everywhere in
// the slab.  The lower chain is convex and the upper chain concave, so over
// a slab's columns [a, b] their extreme values lie at a or at b: ylo =
// max(lower(a), lower(b)) and yhi = min(upper(a), upper(b)), each evaluated
// in float on its edge's line, fmaf(x - x_e, slope_e, y_e) with slope_e =
// dy / dx rounded once, and moved outwards by kPolyMargin = 2048 units.
// The rounding error stays below 512 units: the slope carries at most
// 3.1 x 2^-24 of relative error and x - x_e one more 2^-24, on a product of
// magnitude at most |dy| <= 2^30 (x lies on the edge); y_e (|y_e| <= 2^29)
// is rounded to within 32 units and the fused result (below 2^31) to within
// 128.  So ylo lies above and yhi below the exact chains.  A point with xl < x <
// xr in slab s and ylo < y < yhi is then strictly inside the polygon.  The
// test keeps a few more points than the polygon itself (near steep parts of
// the chains, within one slab), never fewer.
#include "hull_internal.cuh"
#include "kernels.h"

namespace gbh {

namespace {

constexpr int K0_BLOCK = 1024;
constexpr int K0_WARPS = K0_BLOCK / 32;
constexpr int K0_ITEMS = 1;          // sampled points a lane loads at once
constexpr u32 kPolyStride = 1024;    // one point in every kPolyStride is sampled
constexpr int kPolyMargin = 2048;    // units the slab bounds move outwards (> the float error)

// Order-preserving map of a float to an unsigned word.
__device__ __forceinline__ u32 ord_f(float f) {
  const u32 b = __float_as_uint(f);
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}


// Builds the polygon and the slab table (the last block; every thread calls).
__device__ void build_poly(PolyTab* T, const int2* __restrict__ P) {
  __shared__ int s_hx[2 * kPolyDirs + 2], s_hy[2 * kPolyDirs + 2];
  __shared__ int s_k, s_ir, s_ok;
  __shared__ float s_slope[2 * kPolyDirs + 2];
  __shared__ int2 s_yb[kPolySlabs];
  __shared__ int s_px[kPolyDirs], s_py[kPolyDirs];
  __shared__ int s_m;
  if (threadIdx.x < kPolyDirs) {
    // The candidates (one per lane), ranked by (x, y) with one warp: lane l
    // goes to position rank(l) = #{lanes before it in (x, y, lane) order}
    // unless an earlier lane holds the same point.
    const int lane = threadIdx.x;
    const u64 v = *reinterpret_cast<volatile u64*>(&T->best[lane]);
    const bool has = v != 0;
    const int2 p = has ? P[(size_t)(~(u32)v) * kPolyStride] : make_int2(0, 0);
    bool dup = false;
    for (int q = 0; q < 32; ++q) {
      const int qx = __shfl_sync(0xFFFFFFFFu, p.x, q), qy = __shfl_sync(0xFFFFFFFFu, p.y, q);
      const bool qh = __shfl_sync(0xFFFFFFFFu, (int)has, q) != 0;
      dup = dup || (qh && q < lane && qx == p.x && qy == p.y);
    }
    // ranks of distinct points: count only the first of every duplicate group
    const bool keep = has && !dup;
    const u32 km = __ballot_sync(0xFFFFFFFFu, keep);
    int r2 = 0;
    for (int q = 0; q < 32; ++q) {
      const int qx = __shfl_sync(0xFFFFFFFFu, p.x, q), qy = __shfl_sync(0xFFFFFFFFu, p.y, q);
      if (((km >> q) & 1u) && q != lane && (qx < p.x || (qx == p.x && qy < p.y))) ++r2;
    }
    if (keep) { s_px[r2] = p.x; s_py[r2] = p.y; }
    if (lane == 0) s_m = __popc(km);
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    // The convex hull of the m <= 32 sorted distinct candidates, one lane
    // per point.  With d_j = p_i - p_j (j < i) and e_k = p_k - p_i (k > i),
    // all in the half-plane of angles (-90, 90] (sorted and distinct), p_i
    // is a strict lower-hull vertex when the most counter-clockwise d_j is
    // strictly clockwise of the most clockwise e_k (every left slope below
    // every right slope), and a strict upper-hull vertex when the most
    // clockwise d_j is strictly counter-clockwise of the most
    // counter-clockwise e_k; p_0 and p_m-1 end both chains.  The hull,
    // counter-clockwise from p_0: the lower vertices in increasing index,
    // then the upper ones in decreasing index (what Andrew's chain with
    // strict turns gives).
    const int lane = threadIdx.x, m = s_m;
    const int px = lane < m ? s_px[lane] : 0, py = lane < m ? s_py[lane] : 0;
    int ljx = 0, ljy = 0, ujx = 0, ujy = 0, lkx = 0, lky = 0, ukx = 0, uky = 0;
    bool hj = false, hk = false;
    for (int q = 0; q < m; ++q) {
      const int qx = __shfl_sync(0xFFFFFFFFu, px, q), qy = __shfl_sync(0xFFFFFFFFu, py, q);
      if (q < lane) {
        const int dx = px - qx, dy = py - qy;
        if (!hj) { ljx = ujx = dx; ljy = ujy = dy; hj = true; }
        if (cross2(ljx, ljy, dx, dy) > 0) { ljx = dx; ljy = dy; }
        if (cross2(ujx, ujy, dx, dy) < 0) { ujx = dx; ujy = dy; }
      } else if (q > lane) {
        const int ex = qx - px, ey = qy - py;
        if (!hk) { lkx = ukx = ex; lky = uky = ey; hk = true; }
        if (cross2(lkx, lky, ex, ey) < 0) { lkx = ex; lky = ey; }
        if (cross2(ukx, uky, ex, ey) > 0) { ukx = ex; uky = ey; }
      }
    }
    const bool endp = lane == 0 || lane == m - 1;
    const bool lo = lane < m && (endp || cross2(ljx, ljy, lkx, lky) > 0);
    const bool up = lane < m && !endp && cross2(ujx, ujy, ukx, uky) < 0;
    const u32 L = __ballot_sync(0xFFFFFFFFu, lo), U = __ballot_sync(0xFFFFFFFFu, up);
    const int nl = __popc(L);
    const u32 lt = (1u << lane) - 1u, gt = lane == 31 ? 0u : (0xFFFFFFFFu << (lane + 1));
    if (lo) { const int q = __popc(L & lt); s_hx[q] = px; s_hy[q] = py; }
    if (up) { const int q = nl + __popc(U & gt); s_hx[q] = px; s_hy[q] = py; }
    const int xfirst = __shfl_sync(0xFFFFFFFFu, px, 0), xlast = __shfl_sync(0xFFFFFFFFu, px, m > 0 ? m - 1 : 0);
    if (lane == 0) {
      const int k = nl + __popc(U);
      s_k = k;
      s_ir = nl - 1;                       // the rightmost corner ends the lower chain
      s_ok = (k >= 3 && m >= 3 && xlast - xfirst >= 2) ? 1 : 0;
    }
  }
  __syncthreads();
  const int k = s_k, ir = s_ir;
  if (!s_ok) {
    if (threadIdx.x == 0) T->ok = 0;
    return;
  }
  const int xl = s_hx[0], xr = s_hx[ir];
  u32 sh = 0;
  while (((u32)(xr - xl) >> sh) >= (u32)kPolySlabs) ++sh;
  const u32 nslab = ((u32)(xr - xl) >> sh) + 1;
  // Lower chain: corners 0 .. ir, x non-decreasing; at x (xl < x < xr) the
  // active edge (lo, lo + 1) has lo the last corner left of x.  Upper
  // chain: corners ir .. k (k = corner 0 again), x non-increasing; the
  // active edge (lo, lo + 1) has lo the last corner right of x.  Every
  // edge's slope once, in double (vertical edges are never active).
  if (threadIdx.x < (u32)k) {
    const int e = threadIdx.x, en = e + 1 < k ? e + 1 : 0;
    const int dx = s_hx[en] - s_hx[e];
    s_slope[e] = dx != 0 ? (float)(s_hy[en] - s_hy[e]) / (float)dx : 0.0f;
  }
  __syncthreads();
  // Every thread builds a run of consecutive slabs: x only grows along it,
  // so the active lower edge only moves forward and the active upper edge
  // only backward.
  auto hx = [&](int i) { return s_hx[i < k ? i : 0]; };
  const u32 per = (nslab + blockDim.x - 1) / blockDim.x;
  const u32 s_begin = threadIdx.x * per, s_end = min(nslab, s_begin + per);
  int le = 0, ue = k - 1;
  auto lower_at = [&](int x) -> float {       // edge (le, le + 1): x(le) < x <= x(le + 1)
    while (le < ir - 1 && s_hx[le + 1] < x) ++le;
    return fmaf((float)(x - s_hx[le]), s_slope[le], (float)s_hy[le]);
  };
  auto upper_at = [&](int x) -> float {       // edge (ue, ue + 1): x(ue) > x >= x(ue + 1)
    while (ue > ir && hx(ue) <= x) --ue;
    return fmaf((float)(x - s_hx[ue]), s_slope[ue], (float)s_hy[ue]);
  };
  for (u32 s = s_begin; s < s_end; ++s) {
    const long long a0 = (long long)xl + ((long long)s << sh);
    const long long b0 = a0 + ((long long)1 << sh) - 1;
    const int a = (int)(a0 > xl + 1 ? a0 : xl + 1);
    const int b = (int)(b0 < xr - 1 ? b0 : xr - 1);
    int2 yb = make_int2(1, 0);               // empty: nothing strictly inside
    if (a <= b) {
      const float la = lower_at(a), ua = upper_at(a), lb = lower_at(b), ub = upper_at(b);
      const long long lo = (long long)floorf(la > lb ? la : lb) + kPolyMargin;
      const long long hi = (long long)ceilf(ua < ub ? ua : ub) - kPolyMargin;
      if (lo < hi) yb = make_int2((int)lo, (int)hi);
    }
    s_yb[s] = yb;
  }
  __syncthreads();
  for (u32 s = threadIdx.x; s < nslab; s += blockDim.x) T->yb[s] = s_yb[s];
  __syncthreads();
  if (threadIdx.x == 0) {
    T->k = k; T->xl = xl; T->xr = xr; T->sh = sh; T->nslab = nslab;
    T->ok = 1;
  }
}

__global__ void __launch_bounds__(K0_BLOCK)
k0_poly(const int2* __restrict__ P, u32 n, PolyTab* __restrict__ T) {
  __shared__ float s_c[kPolyDirs], s_s[kPolyDirs];
  __shared__ u64 s_best[K0_WARPS][kPolyDirs];
  __shared__ bool s_last;
  if (threadIdx.x < kPolyDirs) {
    float sn, cs;
    sincospif(2.0f * (float)threadIdx.x / (float)kPolyDirs, &sn, &cs);
    s_c[threadIdx.x] = cs;
    s_s[threadIdx.x] = sn;
  }
  __syncthreads();
  const u32 ns = (n + kPolyStride - 1) / kPolyStride;
  // Lane j keeps direction j's largest projection and its sample index; a
  // warp takes 32 K0_ITEMS consecutive samples at a time (every lane loads
  // K0_ITEMS of them at once, then all lanes visit all of them through
  // shuffles, in increasing index: a strict comparison keeps the smallest
  // index among equal projections).
  static_assert(kPolyDirs == 32, "a direction per lane");
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const float cj = s_c[lane], sj = s_s[lane];
  float bp = -3.0e38f;
  u32 bi = 0xFFFFFFFFu;
  const u32 gw = (blockIdx.x * K0_BLOCK + threadIdx.x) >> 5, nw = (gridDim.x * K0_BLOCK) >> 5;
  for (u32 g0 = gw * (32u * K0_ITEMS); g0 < ns; g0 += nw * (32u * K0_ITEMS)) {
    int2 p[K0_ITEMS];
    #pragma unroll
    for (int r = 0; r < K0_ITEMS; ++r) {
      const u32 i = g0 + r * 32u + lane;
      p[r] = i < ns ? P[(size_t)i * kPolyStride] : make_int2(0, 0);
    }
    #pragma unroll
    for (int r = 0; r < K0_ITEMS; ++r) {
      const u32 base = g0 + r * 32u;
      for (int q = 0; q < 32; ++q) {
        const float fx = (float)__shfl_sync(0xFFFFFFFFu, p[r].x, q);
        const float fy = (float)__shfl_sync(0xFFFFFFFFu, p[r].y, q);
        const float v = fmaf(fx, cj, fy * sj);
        if (base + q < ns && v > bp) { bp = v; bi = base + q; }
      }
    }
  }
  s_best[wid][lane] = bi == 0xFFFFFFFFu ? 0ull : (((u64)ord_f(bp) << 32) | (u64)(~bi));
  __syncthreads();
  // The threads that update T->best order their updates before the block's
  // arrival; those of the last block order the arrivals before their reads.
  if (threadIdx.x < kPolyDirs) {
    u64 v = 0;
    for (int w = 0; w < K0_WARPS; ++w) v = s_best[w][threadIdx.x] > v ? s_best[w][threadIdx.x] : v;
    if (v) atomicMax(reinterpret_cast<unsigned long long*>(&T->best[threadIdx.x]), (unsigned long long)v);
    __threadfence();
  }
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(&T->done, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!s_last) return;
  if (threadIdx.x < kPolyDirs) __threadfence();
  build_poly(T, P);
}

}  // namespace

cudaError_t launch_poly(const int* xy, u32 n, PolyTab* T, int num_sms, cudaStream_t st) {
  const u32 ns = (n + kPolyStride - 1) / kPolyStride;
  u32 grid = (ns + K0_BLOCK * K0_ITEMS - 1) / (K0_BLOCK * K0_ITEMS);
  const u32 cap = (u32)num_sms * 2;
  if (grid > cap) grid = cap;
  if (grid < 1) grid = 1;
  k0_poly<<<grid, K0_BLOCK, 0, st>>>(reinterpret_cast<const int2*>(xy), n, T);
  return cudaGetLastError();
}

}  // namespace gbh
