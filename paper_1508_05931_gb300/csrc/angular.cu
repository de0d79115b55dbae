// The paper's own ordering (Section 2.1 steps 3-7, Sections 3.2-3.3): the
// first-round survivors sorted by angle about an anchor, P_longest, and
// Figure 2's two walks as the paper prints them -- forward over the right
// region from P_0, backward over the left region from the last point.
//
// Anchor: P_miny = argmin (y, x, index), so every other point has dy > 0 or
// (dy = 0, dx > 0) and an angle in [0, pi).  The angle is an exact 64-bit
// key: two sector bits (45 degrees each) and floor(t 2^61) of the
// sector-reduced slope t in [0, 1] (reversed where t falls as the angle
// grows).  With |dx|, |dy| <= 2^30 two distinct slopes differ by at least
// 2^-60, so their keys differ and keep their order; equal directions give
// equal keys.  Equal angles are ordered nearer first, then by index: the
// pairs are first sorted by squared distance (ties by index, the input
// order), then stably by angle with each pair's rank in that order as value.
//
// Walks: with L = P_l (the first of the points farthest from P_0, a strict
// vertex) every direction P - L, P != L, lies in an open half-plane, where
// the cross product orders directions totally.  Forward, P_i is kept exactly
// when P_i - L is strictly counter-clockwise of P_temp - L, and P_temp - L is
// the most counter-clockwise direction among P_0 - L and the directions of
// the points before P_i (a point that is not kept does not change it): an
// exclusive prefix maximum.  Backward, P_i is kept exactly when P_i - L is
// strictly clockwise of the most clockwise direction among the points after
// it: an exclusive suffix minimum.  A point equal to L has no direction: it
// is never kept and changes nothing (the walk's test is 0 on it).  Both scans
// run over tiles of AW_TILE positions: per-tile aggregates, one thread
// chaining the tiles, then every tile's positions marked from its carry.
#include "hull_internal.cuh"
#include "kernels.h"

namespace gbh {

namespace {

constexpr int AK_BLOCK = 256;
constexpr int AW_BLOCK = 256;
constexpr int AW_ITEMS = 8;
constexpr int AW_TILE = AW_BLOCK * AW_ITEMS;

// floor(num 2^61 / den) for 0 <= num <= den <= 2^30, den > 0, by two exact
// 64-bit divisions: num 2^61 = (num 2^31) 2^30 and num 2^31 = q1 den + r1.
__device__ __forceinline__ u64 slope_bits(u64 num, u64 den) {
  const u64 hi = num << 31;
  const u64 q1 = hi / den, r1 = hi - q1 * den;
  return (q1 << 30) + (r1 << 30) / den;
}

// The angle key of (dx, dy) != 0 with dy > 0 or (dy == 0, dx > 0).
__device__ __forceinline__ u64 angle_key(long long dx, long long dy) {
  constexpr u64 kOne = 1ull << 61;
  if (dx > 0 && dy <= dx) return slope_bits((u64)dy, (u64)dx);                          // [0, 45]
  if (dx >= 0) return (1ull << 62) | (kOne - slope_bits((u64)dx, (u64)dy));             // (45, 90]
  if (dy >= -dx) return (2ull << 62) | slope_bits((u64)(-dx), (u64)dy);                 // (90, 135]
  return (3ull << 62) | (kOne - slope_bits((u64)dy, (u64)(-dx)));                       // (135, 180)
}

__device__ __forceinline__ u64 dist2(int2 p, int2 o) {
  const long long dx = (long long)p.x - o.x, dy = (long long)p.y - o.y;
  return (u64)(dx * dx + dy * dy);
}

// Pass 1 pairs: (squared distance to the anchor, index) of every first-round
// survivor; n_same counts the points equal to the anchor (distance 0).
__global__ void __launch_bounds__(AK_BLOCK)
k_angle_dist(const int2* __restrict__ xy, const int* __restrict__ keep, u32 s, u32 anchor, u64* __restrict__ keys,
             u32* __restrict__ vals, u32* __restrict__ n_same) {
  const int2 o = xy[anchor];
  u32 same = 0;
  for (u32 j = blockIdx.x * blockDim.x + threadIdx.x; j < s; j += gridDim.x * blockDim.x) {
    const u32 i = (u32)keep[j];
    const u64 d = dist2(xy[i], o);
    keys[j] = d;
    vals[j] = i;
    same += d == 0ull ? 1u : 0u;
  }
  same = __reduce_add_sync(0xFFFFFFFFu, same);
  if ((threadIdx.x & 31) == 0 && same) atomicAdd(n_same, same);
}

// Pass 2 pairs, in pass-1 order: (angle key, rank j); the points equal to
// the anchor get the largest key and sort last.
__global__ void __launch_bounds__(AK_BLOCK)
k_angle_keys(const int2* __restrict__ xy, const u64* __restrict__ dkeys, const u32* __restrict__ dvals, u32 s,
             u32 anchor, u64* __restrict__ keys, u32* __restrict__ vals) {
  const int2 o = xy[anchor];
  for (u32 j = blockIdx.x * blockDim.x + threadIdx.x; j < s; j += gridDim.x * blockDim.x) {
    u64 k = ~0ull;
    if (dkeys[j] != 0ull) {
      const int2 p = xy[dvals[j]];
      k = angle_key((long long)p.x - o.x, (long long)p.y - o.y);
    }
    keys[j] = k;
    vals[j] = j;
  }
}

// order[0] = the anchor, order[k + 1] = the k-th point by angle; pts the
// same points' coordinates.
__global__ void __launch_bounds__(AK_BLOCK)
k_angle_order(const int2* __restrict__ xy, const u32* __restrict__ dvals, const u32* __restrict__ avals, u32 m1,
              u32 anchor, int* __restrict__ order, int2* __restrict__ pts) {
  for (u32 k = blockIdx.x * blockDim.x + threadIdx.x; k < m1; k += gridDim.x * blockDim.x) {
    const u32 i = k == 0 ? anchor : dvals[avals[k - 1]];
    order[k] = (int)i;
    pts[k] = xy[i];
  }
}

// P_l: the largest squared distance to P_0, then the first position holding it.
__global__ void __launch_bounds__(AK_BLOCK) k_angle_lmax(const int2* __restrict__ pts, u32 m1, u64* dmax) {
  const int2 o = pts[0];
  u64 best = 0;
  for (u32 p = 1 + blockIdx.x * blockDim.x + threadIdx.x; p < m1; p += gridDim.x * blockDim.x) {
    const u64 d = dist2(pts[p], o);
    best = d > best ? d : best;
  }
  #pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const u64 v = __shfl_xor_sync(0xFFFFFFFFu, best, off);
    best = v > best ? v : best;
  }
  if ((threadIdx.x & 31) == 0 && best) atomicMax(reinterpret_cast<unsigned long long*>(dmax), (unsigned long long)best);
}

__global__ void __launch_bounds__(AK_BLOCK)
k_angle_lpos(const int2* __restrict__ pts, u32 m1, const u64* __restrict__ dmax, u32* lpos) {
  const int2 o = pts[0];
  const u64 dm = *dmax;
  for (u32 p = 1 + blockIdx.x * blockDim.x + threadIdx.x; p < m1; p += gridDim.x * blockDim.x)
    if (dist2(pts[p], o) == dm) atomicMin(lpos, p);
}

struct Dv {
  int x, y;
  bool v;   // false: no direction yet (the identity)
};

__device__ __forceinline__ long long crs(const Dv& a, const Dv& b) {
  return (long long)a.x * b.y - (long long)a.y * b.x;
}
// The more counter-clockwise (forward walk) / clockwise (backward walk) of
// two directions; equal directions keep the first.
__device__ __forceinline__ Dv more_ccw(const Dv& a, const Dv& b) {
  if (!a.v) return b;
  if (!b.v) return a;
  return crs(a, b) > 0 ? b : a;
}
__device__ __forceinline__ Dv more_cw(const Dv& a, const Dv& b) {
  if (!a.v) return b;
  if (!b.v) return a;
  return crs(a, b) < 0 ? b : a;
}
__device__ __forceinline__ int4 pack_dv(const Dv& a) { return make_int4(a.x, a.y, a.v ? 1 : 0, 0); }
__device__ __forceinline__ Dv unpack_dv(int4 w) { return Dv{w.x, w.y, w.z != 0}; }

// The direction of position p from L (v = false when the point equals L).
__device__ __forceinline__ Dv dir_of(const int2* pts, u32 p, int2 L) {
  const int2 q = pts[p];
  return Dv{q.x - L.x, q.y - L.y, q.x != L.x || q.y != L.y};
}

// This thread's aggregates over its AW_ITEMS positions: forward (1 <= p < l)
// and backward (l < p <= last).
__device__ __forceinline__ void thread_aggs(const int2* pts, u32 m1, u32 l, int2 L, u32 p0, Dv& f, Dv& b) {
  f = Dv{0, 0, false};
  b = Dv{0, 0, false};
  #pragma unroll
  for (int k = 0; k < AW_ITEMS; ++k) {
    const u32 p = p0 + k;
    if (p >= m1 || p == 0 || p == l) continue;
    const Dv d = dir_of(pts, p, L);
    if (!d.v) continue;
    if (p < l) f = more_ccw(f, d);
    else b = more_cw(b, d);
  }
}

__global__ void __launch_bounds__(AW_BLOCK)
k_angle_agg(const int2* __restrict__ pts, u32 m1, const u32* __restrict__ lpos, int4* __restrict__ agg) {
  __shared__ Dv sf[AW_BLOCK], sb[AW_BLOCK];
  const u32 l = *lpos;
  const int2 L = pts[l];
  Dv f, b;
  thread_aggs(pts, m1, l, L, blockIdx.x * AW_TILE + threadIdx.x * AW_ITEMS, f, b);
  sf[threadIdx.x] = f;
  sb[threadIdx.x] = b;
  __syncthreads();
  if (threadIdx.x == 0) {
    Dv a{0, 0, false};
    for (int q = 0; q < AW_BLOCK; ++q) a = more_ccw(a, sf[q]);
    agg[2 * blockIdx.x] = pack_dv(a);
  } else if (threadIdx.x == 32) {
    Dv a{0, 0, false};
    for (int q = 0; q < AW_BLOCK; ++q) a = more_cw(a, sb[q]);
    agg[2 * blockIdx.x + 1] = pack_dv(a);
  }
}

// One thread: each tile's forward carry (P_0 - L and every earlier tile) and
// backward carry (every later tile).
__global__ void k_angle_carry(const int2* __restrict__ pts, const u32* __restrict__ lpos, const int4* __restrict__ agg,
                              u32 nblk, int4* __restrict__ carry) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int2 L = pts[*lpos], P0 = pts[0];
  Dv run{P0.x - L.x, P0.y - L.y, true};
  for (u32 t = 0; t < nblk; ++t) {
    carry[2 * t] = pack_dv(run);
    run = more_ccw(run, unpack_dv(agg[2 * t]));
  }
  Dv rb{0, 0, false};
  for (u32 t = nblk; t-- > 0;) {
    carry[2 * t + 1] = pack_dv(rb);
    rb = more_cw(rb, unpack_dv(agg[2 * t + 1]));
  }
}

__global__ void __launch_bounds__(AW_BLOCK)
k_angle_mark(const int2* __restrict__ pts, u32 m1, const u32* __restrict__ lpos, const int4* __restrict__ carry,
             unsigned char* __restrict__ keep) {
  __shared__ Dv sf[AW_BLOCK], sb[AW_BLOCK];
  const u32 l = *lpos, last = m1 - 1;
  const int2 L = pts[l];
  const u32 p0 = blockIdx.x * AW_TILE + threadIdx.x * AW_ITEMS;
  Dv f, b;
  thread_aggs(pts, m1, l, L, p0, f, b);
  sf[threadIdx.x] = f;
  sb[threadIdx.x] = b;
  __syncthreads();
  if (threadIdx.x == 0) {                 // exclusive prefix over the threads, in place
    Dv run = unpack_dv(carry[2 * blockIdx.x]);
    for (int q = 0; q < AW_BLOCK; ++q) {
      const Dv t = sf[q];
      sf[q] = run;
      run = more_ccw(run, t);
    }
  } else if (threadIdx.x == 32) {         // exclusive suffix
    Dv run = unpack_dv(carry[2 * blockIdx.x + 1]);
    for (int q = AW_BLOCK - 1; q >= 0; --q) {
      const Dv t = sb[q];
      sb[q] = run;
      run = more_cw(run, t);
    }
  }
  __syncthreads();
  Dv run = sf[threadIdx.x];
  #pragma unroll
  for (int k = 0; k < AW_ITEMS; ++k) {
    const u32 p = p0 + k;
    if (p >= m1) break;
    if (p == 0 || p == l || p == last) { keep[p] = 1; continue; }
    if (p > l) continue;                  // the backward walk's
    const Dv d = dir_of(pts, p, L);
    keep[p] = (d.v && crs(run, d) > 0) ? 1 : 0;
    if (d.v) run = more_ccw(run, d);
  }
  run = sb[threadIdx.x];
  #pragma unroll
  for (int k = AW_ITEMS - 1; k >= 0; --k) {
    const u32 p = p0 + k;
    if (p >= m1 || p <= l) continue;
    const Dv d = dir_of(pts, p, L);
    if (p != last) keep[p] = (d.v && (!run.v || crs(run, d) < 0)) ? 1 : 0;
    if (d.v) run = more_cw(run, d);
  }
}

// Step 8 of the angular variant: the kept positions (in any order; sorted
// afterwards), their points and labels in angular order, and the hull's
// positions mapped back to input indices.
__global__ void __launch_bounds__(AK_BLOCK)
k_angle_compact(const unsigned char* __restrict__ keep, u32 m1, u32* __restrict__ pos, u32* __restrict__ cnt) {
  for (u32 p = blockIdx.x * blockDim.x + threadIdx.x; p < m1; p += gridDim.x * blockDim.x)
    if (keep[p]) pos[atomicAdd(cnt, 1u)] = p;
}

__global__ void __launch_bounds__(AK_BLOCK)
k_angle_poskeys(const u32* __restrict__ pos, u32 r, u64* __restrict__ keys, u32* __restrict__ vals) {
  for (u32 j = blockIdx.x * blockDim.x + threadIdx.x; j < r; j += gridDim.x * blockDim.x) {
    keys[j] = pos[j];
    vals[j] = pos[j];
  }
}

__global__ void __launch_bounds__(AK_BLOCK)
k_angle_gather(const int2* __restrict__ xy, const int* __restrict__ order, const u32* __restrict__ spos, u32 r,
               int2* __restrict__ xy_c, int* __restrict__ lab) {
  for (u32 j = blockIdx.x * blockDim.x + threadIdx.x; j < r; j += gridDim.x * blockDim.x) {
    const int i = order[spos[j]];
    xy_c[j] = xy[i];
    lab[j] = i;
  }
}

__global__ void __launch_bounds__(AK_BLOCK)
k_angle_label(const int* __restrict__ out_c, const int* __restrict__ lab, u32 h, int* __restrict__ out) {
  for (u32 k = blockIdx.x * blockDim.x + threadIdx.x; k < h; k += gridDim.x * blockDim.x) out[k] = lab[out_c[k]];
}

int grid_of(u32 n, int num_sms) {
  const u32 g = (n + AK_BLOCK - 1) / AK_BLOCK;
  const u32 cap = (u32)num_sms * 8u;
  return (int)(g < 1u ? 1u : (g < cap ? g : cap));
}

}  // namespace

cudaError_t launch_angle_dist(const int2* xy, const int* keep, u32 s, u32 anchor, u64* keys, u32* vals, u32* n_same,
                              int num_sms, cudaStream_t st) {
  k_angle_dist<<<grid_of(s, num_sms), AK_BLOCK, 0, st>>>(xy, keep, s, anchor, keys, vals, n_same);
  return cudaGetLastError();
}

cudaError_t launch_angle_keys(const int2* xy, const u64* dkeys, const u32* dvals, u32 s, u32 anchor, u64* keys,
                              u32* vals, int num_sms, cudaStream_t st) {
  k_angle_keys<<<grid_of(s, num_sms), AK_BLOCK, 0, st>>>(xy, dkeys, dvals, s, anchor, keys, vals);
  return cudaGetLastError();
}

cudaError_t launch_angle_order(const int2* xy, const u32* dvals, const u32* avals, u32 m1, u32 anchor, int* order,
                               int2* pts, int num_sms, cudaStream_t st) {
  k_angle_order<<<grid_of(m1, num_sms), AK_BLOCK, 0, st>>>(xy, dvals, avals, m1, anchor, order, pts);
  return cudaGetLastError();
}

cudaError_t launch_angle_compact(const unsigned char* keep, u32 m1, u32* pos, u32* cnt, int num_sms, cudaStream_t st) {
  k_angle_compact<<<grid_of(m1, num_sms), AK_BLOCK, 0, st>>>(keep, m1, pos, cnt);
  return cudaGetLastError();
}

cudaError_t launch_angle_gather(const int2* xy, const int* order, u32* pos, u32 r, u64* keys, u32* vals, int2* xy_c,
                                int* lab, int num_sms, cudaStream_t st, int phase) {
  if (phase == 0) {
    k_angle_poskeys<<<grid_of(r, num_sms), AK_BLOCK, 0, st>>>(pos, r, keys, vals);
  } else {
    k_angle_gather<<<grid_of(r, num_sms), AK_BLOCK, 0, st>>>(xy, order, vals, r, xy_c, lab);
  }
  return cudaGetLastError();
}

cudaError_t launch_angle_label(const int* out_c, const int* lab, u32 h, int* out, int num_sms, cudaStream_t st) {
  k_angle_label<<<grid_of(h, num_sms), AK_BLOCK, 0, st>>>(out_c, lab, h, out);
  return cudaGetLastError();
}

size_t angle_walk_scratch_bytes(u32 m1) {
  const size_t nblk = ((size_t)m1 + AW_TILE - 1) / AW_TILE;
  return 16 + nblk * 4 * sizeof(int4);
}

cudaError_t launch_angle_walks(const int2* pts, u32 m1, void* scratch, u32* lpos, unsigned char* keep, int num_sms,
                               cudaStream_t st) {
  u64* dmax = reinterpret_cast<u64*>(scratch);
  int4* agg = reinterpret_cast<int4*>(reinterpret_cast<char*>(scratch) + 16);
  const u32 nblk = (m1 + AW_TILE - 1) / AW_TILE;
  cudaError_t e = cudaMemsetAsync(dmax, 0, 8, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(lpos, 0xFF, 4, st);
  if (e != cudaSuccess) return e;
  k_angle_lmax<<<grid_of(m1, num_sms), AK_BLOCK, 0, st>>>(pts, m1, dmax);
  k_angle_lpos<<<grid_of(m1, num_sms), AK_BLOCK, 0, st>>>(pts, m1, dmax, lpos);
  k_angle_agg<<<nblk, AW_BLOCK, 0, st>>>(pts, m1, lpos, agg);
  k_angle_carry<<<1, 32, 0, st>>>(pts, lpos, agg, nblk, agg + 2 * nblk);
  k_angle_mark<<<nblk, AW_BLOCK, 0, st>>>(pts, m1, lpos, agg + 2 * nblk, keep);
  return cudaGetLastError();
}

}  // namespace gbh
