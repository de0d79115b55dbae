// K4: region split and the second-round filter (Section 2.1 steps 5-7,
// Section 2.2 / Figure 2, Section 3.4), fused with the stable compaction
// that Section 3.4 performs with a stable partition.
//
// Over the sorted survivors: P_0 = P_minx (first in the lexicographic
// order) and P_l = P_maxx (the last distinct point, its smallest index).
// A point strictly right of the directed line P_0 -> P_l belongs to the
// lower region, strictly left to the upper region; points on the line are
// dropped.  Figure 2 walks a region with a running P_temp and discards P_i
// when it lies left of (right of, for the upper region) or on the line
// P_temp -> P_l.  With d(p) = p - P_l, that rule keeps P_i exactly when
// d(P_i) is strictly counter-clockwise (clockwise) of d(P_temp), and P_temp
// is always the point with the extreme direction seen so far, starting from
// d(P_0).  All directions of a region lie in one half-plane, where the
// cross product orders them totally, so "extreme so far" is an exclusive
// prefix max (min) -- an associative scan -- and gives exactly the
// survivors of the sequential loop; duplicates of a kept point fall out as
// equal directions.
//
// One pass over chunks of K4_CHUNK sorted points, taken in order through a
// dynamic chunk id:
//   k4_scan     per chunk: the extreme directions of each thread's points,
//               of each warp and of the chunk (published at once), the
//               exclusive prefix over earlier chunks by a decoupled
//               look-back (one warp, 32 chunks per step, bounded waits; the
//               operation is a maximum under a total order, so partial
//               results combine in any order), then the keep decisions, the
//               kept points staged per chunk and the per-chunk kept counts;
//               the last block scans the counts into offsets and adds P_0
//               and P_l to both region lists;
//   k4_compact  moves the few kept points into the region lists in order.
#include "hull_internal.cuh"
#include "kernels.h"
#include "regions.cuh"

namespace gbh {

namespace {

#ifndef K4_BLOCK_CFG
#define K4_BLOCK_CFG 256
#endif
constexpr int K4_BLOCK = K4_BLOCK_CFG;
constexpr int K4_ITEMS = 8;
constexpr int K4_CHUNK = K4_BLOCK * K4_ITEMS;      // sorted points per chunk
constexpr int K4_WARPS = K4_BLOCK / 32;

struct Geo {
  const u64* keys;
  const u32* idxs;
  u32 s, ybits;
  u64 ymask;
  int x0, y0, ax, ay, bx, by, ux, uy, d0x, d0y;
};

__device__ __forceinline__ Geo make_geo(const Plan* plan, const u64* ka, const u32* ia,
                                        const u64* kb, const u32* ib) {
  Geo g;
  // Buffer a holds the result after an even number of radix passes, b
  // after an odd number or after the bucket sort.
  const bool in_b = plan->sorted_in_b != 0;
  g.keys = in_b ? kb : ka;
  g.idxs = in_b ? ib : ia;
  g.s = plan->s;
  g.ybits = plan->ybits;
  g.ymask = g.ybits ? ((~0ull) >> (64 - g.ybits)) : 0ull;
  g.x0 = plan->key_x0; g.y0 = plan->key_y0;
  g.ax = plan->ext_x[0]; g.ay = plan->ext_y[0];     // P_0 = P_minx
  g.bx = plan->ext_x[1]; g.by = plan->ext_y[1];     // P_l = P_maxx
  g.ux = g.bx - g.ax; g.uy = g.by - g.ay;
  g.d0x = g.ax - g.bx; g.d0y = g.ay - g.by;         // d(P_0)
  return g;
}

// Loads this thread's K4_ITEMS consecutive sorted points and classifies them.
__device__ __forceinline__ void load_items(const Geo& g, u32 first, int* px, int* py, int* pi,
                                           signed char* side, bool with_idx) {
  u64 kk[K4_ITEMS];
  if (first + K4_ITEMS <= g.s) {
    const ulonglong2* kp = reinterpret_cast<const ulonglong2*>(g.keys + first);
    #pragma unroll
    for (int v = 0; v < K4_ITEMS / 2; ++v) { const ulonglong2 q = kp[v]; kk[2 * v] = q.x; kk[2 * v + 1] = q.y; }
    if (with_idx) {
      const int4* ip = reinterpret_cast<const int4*>(g.idxs + first);
      #pragma unroll
      for (int v = 0; v < K4_ITEMS / 4; ++v) {
        const int4 q = ip[v];
        pi[4 * v] = q.x; pi[4 * v + 1] = q.y; pi[4 * v + 2] = q.z; pi[4 * v + 3] = q.w;
      }
    }
  } else {
    #pragma unroll
    for (int i = 0; i < K4_ITEMS; ++i) {
      const u32 p = first + i;
      kk[i] = p < g.s ? g.keys[p] : 0ull;
      if (with_idx) pi[i] = p < g.s ? (int)g.idxs[p] : 0;
    }
  }
  #pragma unroll
  for (int i = 0; i < K4_ITEMS; ++i) {
    px[i] = g.x0 + (int)(u32)(kk[i] >> g.ybits);
    py[i] = g.y0 + (int)(u32)(kk[i] & g.ymask);
    const long long o = cross2(g.ux, g.uy, px[i] - g.ax, py[i] - g.ay);
    side[i] = (first + i >= g.s) ? 0 : ((o < 0) ? -1 : (o > 0 ? 1 : 0));
  }
}

__device__ __forceinline__ Dir2 thread_agg(const Geo& g, const int* px, const int* py,
                                           const signed char* side) {
  Dir2 a = {g.d0x, g.d0y, g.d0x, g.d0y};
  #pragma unroll
  for (int i = 0; i < K4_ITEMS; ++i) {
    if (side[i] < 0) cmax(a.lx, a.ly, px[i] - g.bx, py[i] - g.by);
    else if (side[i] > 0) cmin(a.ux, a.uy, px[i] - g.bx, py[i] - g.by);
  }
  return a;
}

__global__ void __launch_bounds__(K4_BLOCK, 1024 / K4_BLOCK)
k4_scan(const u64* __restrict__ ka, const u32* __restrict__ ia, const u64* __restrict__ kb,
        const u32* __restrict__ ib, Plan* plan, K4Chunk* __restrict__ chunks,
        int2* __restrict__ t_lo_xy, int* __restrict__ t_lo_idx, int2* __restrict__ t_up_xy,
        int* __restrict__ t_up_idx, int2* __restrict__ lo_xy, int* __restrict__ lo_idx,
        int2* __restrict__ up_xy, int* __restrict__ up_idx) {
  __shared__ Dir2 s_w[K4_WARPS];
  __shared__ Dir2 s_excl;
  __shared__ u32 s_wc[K4_WARPS][2];
  __shared__ u32 s_chunk;
  __shared__ int s_fail;
  __shared__ bool s_last;
  if (plan->error & (ERR_RANGE | ERR_FALLBACK)) return;
  const Geo g = make_geo(plan, ka, ia, kb, ib);
  const u32 nchunks = (g.s + K4_CHUNK - 1) / K4_CHUNK;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const u32 spin = plan->spin_limit;
  const Dir2 ident = {g.d0x, g.d0y, g.d0x, g.d0y};
  bool failed = false;
  for (;;) {
    if (threadIdx.x == 0) s_chunk = atomicAdd(&plan->ctr[CTR_REGION], 1u);
    __syncthreads();
    const u32 c = s_chunk;
    if (c >= nchunks) break;
    int px[K4_ITEMS], py[K4_ITEMS], pi[K4_ITEMS];
    signed char side[K4_ITEMS];
    load_items(g, c * K4_CHUNK + threadIdx.x * K4_ITEMS, px, py, pi, side, true);
    const Dir2 agg = thread_agg(g, px, py, side);
    const Dir2 inc = warp_scan_dir(agg);
    Dir2 lex = shfl_up_dir(inc, 1);
    if (lane == 31) s_w[wid] = inc;
    __syncthreads();
    // Warp 0: publish the chunk aggregate, look back, publish the prefix.
    if (wid == 0) {
      Dir2 t = ident;
      #pragma unroll
      for (int w = 0; w < K4_WARPS; ++w) combine(t, s_w[w]);
      K4Chunk* ch = &chunks[c];
      if (lane == 0) {
        st_relaxed_u64(c == 0 ? &ch->inc_lo : &ch->agg_lo, pack_dir(t.lx, t.ly));
        st_relaxed_u64(c == 0 ? &ch->inc_up : &ch->agg_up, pack_dir(t.ux, t.uy));
      }
      Dir2 excl = ident;
      bool ok = true;
      if (c > 0) ok = lookback_dir(chunks, c, plan, spin, ident, &excl);
      if (lane == 0) {
        s_fail = ok ? 0 : 1;
        s_excl = excl;
        if (ok && c > 0) {
          Dir2 in = excl;
          combine(in, t);
          st_relaxed_u64(&ch->inc_lo, pack_dir(in.lx, in.ly));
          st_relaxed_u64(&ch->inc_up, pack_dir(in.ux, in.uy));
        }
      }
    }
    __syncthreads();
    if (s_fail) { failed = true; break; }
    Dir2 run = s_excl;
    for (int w = 0; w < wid; ++w) combine(run, s_w[w]);
    if (lane > 0) combine(run, lex);
    unsigned keep_lo = 0, keep_up = 0;
    #pragma unroll
    for (int i = 0; i < K4_ITEMS; ++i) {
      const int vx = px[i] - g.bx, vy = py[i] - g.by;
      if (side[i] < 0) {
        if (cross2(run.lx, run.ly, vx, vy) > 0) { keep_lo |= 1u << i; run.lx = vx; run.ly = vy; }
      } else if (side[i] > 0) {
        if (cross2(run.ux, run.uy, vx, vy) < 0) { keep_up |= 1u << i; run.ux = vx; run.uy = vy; }
      }
    }
    // Stable ranks of the kept points inside the chunk.
    const u32 c_lo = __popc(keep_lo), c_up = __popc(keep_up);
    u32 i_lo = c_lo, i_up = c_up;
    #pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const u32 t0 = __shfl_up_sync(0xFFFFFFFFu, i_lo, o);
      const u32 t1 = __shfl_up_sync(0xFFFFFFFFu, i_up, o);
      if (lane >= o) { i_lo += t0; i_up += t1; }
    }
    if (lane == 31) { s_wc[wid][0] = i_lo; s_wc[wid][1] = i_up; }
    __syncthreads();
    u32 wl = 0, wu = 0, tl = 0, tu = 0;
    for (int w = 0; w < K4_WARPS; ++w) {
      if (w < wid) { wl += s_wc[w][0]; wu += s_wc[w][1]; }
      tl += s_wc[w][0]; tu += s_wc[w][1];
    }
    if (threadIdx.x == 0) { chunks[c].cnt = make_uint2(tl, tu); chunks[c].base = c * K4_CHUNK; }
    u32 pl = c * K4_CHUNK + wl + i_lo - c_lo;
    u32 pu = c * K4_CHUNK + wu + i_up - c_up;
    #pragma unroll
    for (int i = 0; i < K4_ITEMS; ++i) {
      if (keep_lo & (1u << i)) { t_lo_xy[pl] = make_int2(px[i], py[i]); t_lo_idx[pl] = pi[i]; ++pl; }
      else if (keep_up & (1u << i)) { t_up_xy[pu] = make_int2(px[i], py[i]); t_up_idx[pu] = pi[i]; ++pu; }
    }
    __syncthreads();
  }
  if (failed) return;
  if (!last_block(plan, CTR_REGION2, &s_last)) return;
  region_offsets(plan, chunks, nchunks, g.s, &s_wc[0][0], lo_xy, lo_idx, up_xy, up_idx);
}

// Moves the kept points staged per record (from slot base) into the region
// lists in order.  Records: K4's chunks, or the bucket sort's groups
// (GROUPS: their number is plan->ngroups).
template <bool GROUPS>
__global__ void __launch_bounds__(K4_BLOCK)
k4_compact(Plan* plan, const K4Chunk* __restrict__ chunks, const int2* __restrict__ t_lo_xy,
           const int* __restrict__ t_lo_idx, const int2* __restrict__ t_up_xy,
           const int* __restrict__ t_up_idx, int2* __restrict__ lo_xy, int* __restrict__ lo_idx,
           int2* __restrict__ up_xy, int* __restrict__ up_idx) {
  if (plan->error & (ERR_RANGE | ERR_TIMEOUT | ERR_FALLBACK)) return;
  const u32 s = plan->s;
  const u32 nrec = GROUPS ? plan->ngroups : (s + K4_CHUNK - 1) / K4_CHUNK;
  for (u32 c = blockIdx.x; c < nrec; c += gridDim.x) {
    const uint2 cnt = chunks[c].cnt, off = chunks[c].off;
    const u32 base = chunks[c].base;
    for (u32 j = threadIdx.x; j < cnt.x; j += K4_BLOCK) {
      const u32 d = 1 + off.x + j;
      if (d < s + 1 && base + j < s) { lo_xy[d] = t_lo_xy[base + j]; lo_idx[d] = t_lo_idx[base + j]; }
      else flag_error(plan, ERR_INTERNAL);
    }
    for (u32 j = threadIdx.x; j < cnt.y; j += K4_BLOCK) {
      const u32 d = 1 + off.y + j;
      if (d < s + 1 && base + j < s) { up_xy[d] = t_up_xy[base + j]; up_idx[d] = t_up_idx[base + j]; }
      else flag_error(plan, ERR_INTERNAL);
    }
  }
}

}  // namespace

int k4_tile() { return K4_CHUNK; }
size_t k4_status_bytes() { return sizeof(K4Chunk); }

cudaError_t k4_occupancy(int* blocks) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, k4_scan, K4_BLOCK, 0);
}

// `status` holds one K4Chunk per chunk, `nrec` >= ceil(s / K4_CHUNK) of
// them (cleared here); t_* are staging areas of at least nrec * K4_CHUNK
// slots each.
cudaError_t launch_k4(const u64* ka, const u32* ia, const u64* kb, const u32* ib, Plan* plan,
                      void* status, size_t nrec, int2* lo_xy, int* lo_idx, int2* up_xy, int* up_idx,
                      int2* t_lo_xy, int* t_lo_idx, int2* t_up_xy, int* t_up_idx, int grid,
                      cudaStream_t st) {
  K4Chunk* ch = reinterpret_cast<K4Chunk*>(status);
  cudaError_t e = cudaMemsetAsync(status, 0, nrec * sizeof(K4Chunk), st);
  if (e != cudaSuccess) return e;
  k4_scan<<<grid, K4_BLOCK, 0, st>>>(ka, ia, kb, ib, plan, ch, t_lo_xy, t_lo_idx, t_up_xy, t_up_idx,
                                     lo_xy, lo_idx, up_xy, up_idx);
  k4_compact<false><<<grid, K4_BLOCK, 0, st>>>(plan, ch, t_lo_xy, t_lo_idx, t_up_xy, t_up_idx, lo_xy, lo_idx,
                                               up_xy, up_idx);
  return cudaGetLastError();
}

// The mirrored second round (Section 2.2, Figure 2 reflected through
// x -> -x) over both region lists, one block each: L[0] = P_0, L[1..m] the
// forward survivors in sorted order, L[m + 1] = P_l.  The walk goes from
// P_l back to P_0 with directions d = p - P_0 (a half-plane: a total order
// under the cross product); a point is kept when its direction is strictly
// clockwise (lower region) / counter-clockwise (upper) of the running
// extreme, which starts at P_l - P_0: the exclusive prefix extreme of a scan
// in walk order, so the block scans it.  Thread t takes walk positions
// [t R, t R + R) (walk position w is list position m - w).  The kept points
// go to `stage` in ascending list order and then back over L[1..], P_l
// after them; r_lo / r_up become the kept counts.
constexpr int KR_BLOCK = 1024;
constexpr int KR_WARPS = KR_BLOCK / 32;

struct Dir1 {
  int x, y;
};

// b strictly beyond a: clockwise of it for the lower region (sgn > 0),
// counter-clockwise for the upper.
__device__ __forceinline__ bool rev_beyond(const Dir1& a, const Dir1& b, int sgn) {
  const long long c = cross2(a.x, a.y, b.x, b.y);
  return sgn > 0 ? c < 0 : c > 0;
}

constexpr int KR_RB = 8;   // list entries a thread loads at once

// Combination in walk order (a before b): the extreme of the two.
__device__ __forceinline__ Dir1 rev_combine(const Dir1& a, const Dir1& b, int sgn) {
  return rev_beyond(a, b, sgn) ? b : a;
}

__device__ __forceinline__ Dir1 shfl_up_dir1(const Dir1& v, int o) {
  return Dir1{__shfl_up_sync(0xFFFFFFFFu, v.x, o), __shfl_up_sync(0xFFFFFFFFu, v.y, o)};
}

__global__ void __launch_bounds__(KR_BLOCK)
k4_reverse(Plan* plan, int2* lo_xy, int* lo_idx, int2* up_xy, int* up_idx, int2* st_lo_xy, int* st_lo_idx,
           int2* st_up_xy, int* st_up_idx) {
  __shared__ Dir1 s_d[KR_WARPS];
  __shared__ u32 s_c[KR_WARPS];
  if (plan->error & (ERR_RANGE | ERR_TIMEOUT | ERR_INTERNAL | ERR_FALLBACK)) return;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int region = blockIdx.x;
  const int sgn = region == 0 ? 1 : -1;
  int2* L = region == 0 ? lo_xy : up_xy;
  int* LI = region == 0 ? lo_idx : up_idx;
  int2* SX = region == 0 ? st_lo_xy : st_up_xy;
  int* SI = region == 0 ? st_lo_idx : st_up_idx;
  const u32 m = region == 0 ? plan->r_lo : plan->r_up;
  if (m == 0) return;
  const int2 p0 = L[0], pl = L[m + 1];
  const Dir1 u0{pl.x - p0.x, pl.y - p0.y};
  const u32 R = (m + KR_BLOCK - 1) / KR_BLOCK;
  const u32 w0 = min(m, threadIdx.x * R), w1 = min(m, w0 + R);
  // The thread's extreme (it starts at u0, which every combination absorbs).
  Dir1 loc = u0;
  for (u32 wb = w0; wb < w1; wb += KR_RB) {
    int2 q[KR_RB];
    #pragma unroll
    for (int k = 0; k < KR_RB; ++k) q[k] = wb + k < w1 ? L[m - (wb + k)] : p0;
    #pragma unroll
    for (int k = 0; k < KR_RB; ++k)
      if (wb + k < w1) loc = rev_combine(loc, Dir1{q[k].x - p0.x, q[k].y - p0.y}, sgn);
  }
  // Its exclusive prefix: warp scan, then every warp scans the warps' totals.
  Dir1 inc = loc;
  #pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const Dir1 t = shfl_up_dir1(inc, o);
    if (lane >= o) inc = rev_combine(t, inc, sgn);
  }
  const Dir1 lex = shfl_up_dir1(inc, 1);
  if (lane == 31) s_d[wid] = inc;
  __syncthreads();
  Dir1 wi = s_d[lane];
  #pragma unroll
  for (int o = 1; o < KR_WARPS; o <<= 1) {
    const Dir1 t = shfl_up_dir1(wi, o);
    if (lane >= o) wi = rev_combine(t, wi, sgn);
  }
  const Dir1 wprev{__shfl_sync(0xFFFFFFFFu, wi.x, wid > 0 ? wid - 1 : 0),
                   __shfl_sync(0xFFFFFFFFu, wi.y, wid > 0 ? wid - 1 : 0)};
  Dir1 ex = wid > 0 ? wprev : u0;
  if (lane > 0) ex = rev_combine(ex, lex, sgn);
  // Kept points of this thread, then their exclusive count in walk order.
  u32 cnt = 0;
  {
    Dir1 prev = ex;
    for (u32 wb = w0; wb < w1; wb += KR_RB) {
      int2 q[KR_RB];
      #pragma unroll
      for (int k = 0; k < KR_RB; ++k) q[k] = wb + k < w1 ? L[m - (wb + k)] : p0;
      #pragma unroll
      for (int k = 0; k < KR_RB; ++k) {
        const Dir1 d{q[k].x - p0.x, q[k].y - p0.y};
        if (wb + k < w1 && rev_beyond(prev, d, sgn)) { ++cnt; prev = d; }
      }
    }
  }
  u32 ci = cnt;
  #pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const u32 t = __shfl_up_sync(0xFFFFFFFFu, ci, o);
    if (lane >= o) ci += t;
  }
  if (lane == 31) s_c[wid] = ci;
  __syncthreads();
  u32 wc = s_c[lane];
  #pragma unroll
  for (int o = 1; o < KR_WARPS; o <<= 1) {
    const u32 t = __shfl_up_sync(0xFFFFFFFFu, wc, o);
    if (lane >= o) wc += t;
  }
  const u32 total = __shfl_sync(0xFFFFFFFFu, wc, KR_WARPS - 1);
  const u32 wbefore = __shfl_sync(0xFFFFFFFFu, wc, wid > 0 ? wid - 1 : 0);
  const u32 before = (wid > 0 ? wbefore : 0u) + ci - cnt;
  // The kept points in ascending list order (reverse of the walk).
  {
    Dir1 prev = ex;
    u32 k = before;
    for (u32 wb = w0; wb < w1; wb += KR_RB) {
      int2 q[KR_RB];
      #pragma unroll
      for (int j = 0; j < KR_RB; ++j) q[j] = wb + j < w1 ? L[m - (wb + j)] : p0;
      #pragma unroll
      for (int j = 0; j < KR_RB; ++j) {
        const Dir1 d{q[j].x - p0.x, q[j].y - p0.y};
        if (wb + j < w1 && rev_beyond(prev, d, sgn)) {
          const u32 out = total - 1 - k;
          if (out < m) { SX[out] = q[j]; SI[out] = LI[m - (wb + j)]; } else flag_error(plan, ERR_INTERNAL);
          ++k;
          prev = d;
        }
      }
    }
  }
  __syncthreads();
  for (u32 q = threadIdx.x; q < total; q += KR_BLOCK) {
    L[1 + q] = SX[q];
    LI[1 + q] = SI[q];
  }
  if (threadIdx.x == 0) {
    const int pli = LI[m + 1];
    L[total + 1] = pl;
    LI[total + 1] = pli;
    if (region == 0) plan->r_lo = total; else plan->r_up = total;
  }
}

// Section 3.4's chunked second round, as the paper runs it: one block of
// KC_BLOCK threads per region (blockIdx.x 0 lower, 1 upper) over a list
// sorted by (x, y, index): P_l is the first of the list's last run of
// equal points; the region's positions are collected in order into `pos`;
// they are split into bs runs of ceil(m_region / bs) consecutive points and
// thread t < bs checks run t with Figure 2 from P_temp = P_0, in sequence;
// the labels of the kept points go to `out` in list order and their count
// to plan->r_lo / r_up.
constexpr int KC_BLOCK = 1024;
constexpr int KC_WARPS = KC_BLOCK / 32;

__device__ __forceinline__ u32 block_excl_sum(u32 v, u32* red, u32* total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  u32 inc = v;
  #pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const u32 t = __shfl_up_sync(0xFFFFFFFFu, inc, o);
    if (lane >= o) inc += t;
  }
  if (lane == 31) red[wid] = inc;
  __syncthreads();
  u32 w = red[lane < KC_WARPS ? lane : 0];
  if (lane >= KC_WARPS) w = 0;
  #pragma unroll
  for (int o = 1; o < KC_WARPS; o <<= 1) {
    const u32 t = __shfl_up_sync(0xFFFFFFFFu, w, o);
    if (lane >= o) w += t;
  }
  *total = __shfl_sync(0xFFFFFFFFu, w, KC_WARPS - 1);
  const u32 before = __shfl_sync(0xFFFFFFFFu, w, wid > 0 ? wid - 1 : 0);
  __syncthreads();
  return (wid > 0 ? before : 0u) + inc - v;
}

__global__ void __launch_bounds__(KC_BLOCK)
k4_chunked(const int2* __restrict__ xy, const int* __restrict__ idx, u32 m, u32 bs, Plan* plan, int* pos_lo,
           int* pos_up, int* out_lo, int* out_up) {
  __shared__ u32 s_red[KC_WARPS];
  __shared__ u32 s_l;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int region = blockIdx.x;
  int* pos = region == 0 ? pos_lo : pos_up;
  int* out = region == 0 ? out_lo : out_up;
  // P_l: one past the last point that differs from the list's last point.
  const int2 last = xy[m - 1];
  u32 jl = 0;
  for (u32 i = threadIdx.x; i < m; i += KC_BLOCK)
    if (xy[i].x != last.x || xy[i].y != last.y) jl = max(jl, i + 1);
  #pragma unroll
  for (int o = 16; o > 0; o >>= 1) jl = max(jl, __shfl_xor_sync(0xFFFFFFFFu, jl, o));
  if (threadIdx.x == 0) s_l = 0;
  __syncthreads();
  if (lane == 0) atomicMax(&s_l, jl);
  __syncthreads();
  const u32 l = s_l;
  const int2 p0 = xy[0], pl = xy[l];
  if (p0.x == pl.x && p0.y == pl.y) {
    if (threadIdx.x == 0) { if (region == 0) plan->r_lo = 0; else plan->r_up = 0; }
    return;
  }
  // The region's list positions, in order.
  const u32 n1 = m - 1;
  const u32 R = (n1 + KC_BLOCK - 1) / KC_BLOCK;
  const u32 a0 = 1 + min(n1, threadIdx.x * R), a1 = 1 + min(n1, threadIdx.x * R + R);
  const int ux = pl.x - p0.x, uy = pl.y - p0.y;
  auto in_region = [&](const int2 p) {
    const long long sd = cross2(ux, uy, p.x - p0.x, p.y - p0.y);
    return region == 0 ? sd < 0 : sd > 0;
  };
  u32 c = 0;
  for (u32 i = a0; i < a1; ++i) c += in_region(xy[i]) ? 1u : 0u;
  u32 mr;
  u32 o = block_excl_sum(c, s_red, &mr);
  for (u32 i = a0; i < a1; ++i)
    if (in_region(xy[i])) pos[o++] = (int)i;
  __syncthreads();
  // Runs of ceil(mr / bs) positions, Figure 2 over each from P_temp = P_0.
  const u32 run = (mr + bs - 1) / bs;
  const u32 r0 = threadIdx.x < bs ? min(mr, threadIdx.x * run) : mr;
  const u32 r1 = threadIdx.x < bs ? min(mr, r0 + run) : mr;
  auto kept = [&](int2& t, const int2 p) {
    const long long ov = cross2(pl.x - t.x, pl.y - t.y, p.x - t.x, p.y - t.y);
    const bool k = region == 0 ? ov < 0 : ov > 0;
    if (k) t = p;
    return k;
  };
  u32 kc = 0;
  {
    int2 t = p0;
    for (u32 k = r0; k < r1; ++k) kc += kept(t, xy[pos[k]]) ? 1u : 0u;
  }
  u32 total;
  u32 q = block_excl_sum(kc, s_red, &total);
  {
    int2 t = p0;
    for (u32 k = r0; k < r1; ++k) {
      const int i = pos[k];
      if (kept(t, xy[i])) out[q++] = idx[i];
    }
  }
  if (threadIdx.x == 0) { if (region == 0) plan->r_lo = total; else plan->r_up = total; }
}

cudaError_t launch_k4_chunked(const int2* xy, const int* idx, u32 m, u32 bs, Plan* plan, int* pos_lo, int* pos_up,
                              int* out_lo, int* out_up, cudaStream_t st) {
  k4_chunked<<<2, KC_BLOCK, 0, st>>>(xy, idx, m, bs, plan, pos_lo, pos_up, out_lo, out_up);
  return cudaGetLastError();
}

cudaError_t launch_k4_reverse(Plan* plan, int2* lo_xy, int* lo_idx, int2* up_xy, int* up_idx, int2* st_lo_xy,
                              int* st_lo_idx, int2* st_up_xy, int* st_up_idx, cudaStream_t st) {
  k4_reverse<<<2, KR_BLOCK, 0, st>>>(plan, lo_xy, lo_idx, up_xy, up_idx, st_lo_xy, st_lo_idx, st_up_xy, st_up_idx);
  return cudaGetLastError();
}

// The compaction after the bucket sort's fused second round (one record per group).
cudaError_t launch_group_compact(Plan* plan, const void* status, const int2* t_lo_xy, const int* t_lo_idx,
                                 const int2* t_up_xy, const int* t_up_idx, int2* lo_xy, int* lo_idx,
                                 int2* up_xy, int* up_idx, int grid, cudaStream_t st) {
  k4_compact<true><<<grid, K4_BLOCK, 0, st>>>(plan, reinterpret_cast<const K4Chunk*>(status), t_lo_xy, t_lo_idx,
                                              t_up_xy, t_up_idx, lo_xy, lo_idx, up_xy, up_idx);
  return cudaGetLastError();
}

}  // namespace gbh
