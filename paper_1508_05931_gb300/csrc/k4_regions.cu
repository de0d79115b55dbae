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

namespace gbh {

namespace {

#ifndef K4_BLOCK_CFG
#define K4_BLOCK_CFG 256
#endif
constexpr int K4_BLOCK = K4_BLOCK_CFG;
constexpr int K4_ITEMS = 8;
constexpr int K4_CHUNK = K4_BLOCK * K4_ITEMS;      // sorted points per chunk
constexpr int K4_WARPS = K4_BLOCK / 32;

// Extreme directions seen so far: lower region (counter-clockwise-most)
// and upper region (clockwise-most).  d(P_0) is the identity of both
// operations: every lower direction is strictly counter-clockwise of it and
// every upper direction strictly clockwise, so no "empty" case exists.
struct __align__(16) Dir2 {
  int lx, ly, ux, uy;
};

// Look-back words: one direction per word, with a valid bit, so that a
// single 64-bit load both finds and reads a published value.  Every
// direction here has dx <= 0 (P_l has the largest x), so -dx takes 31 bits
// and dy + 2^30 takes 32.  The words are cleared before each call.
struct __align__(64) K4Chunk {
  u64 agg_lo, agg_up;     // chunk aggregate (lower, upper region)
  u64 inc_lo, inc_up;     // inclusive prefix through this chunk (with d(P_0))
  uint2 cnt;              // kept points (lower, upper)
  uint2 off;              // exclusive offsets of the same
  u64 pad[2];
};
static_assert(sizeof(K4Chunk) == 64, "chunk record size");

// Lower region: keep the counter-clockwise-most direction (ties keep a).
__device__ __forceinline__ void cmax(int& ax, int& ay, int bx, int by) {
  const bool t = cross2(ax, ay, bx, by) > 0;
  ax = t ? bx : ax;
  ay = t ? by : ay;
}
// Upper region: keep the clockwise-most direction (ties keep a).
__device__ __forceinline__ void cmin(int& ax, int& ay, int bx, int by) {
  const bool t = cross2(ax, ay, bx, by) < 0;
  ax = t ? bx : ax;
  ay = t ? by : ay;
}
__device__ __forceinline__ void combine(Dir2& a, const Dir2& b) {
  cmax(a.lx, a.ly, b.lx, b.ly);
  cmin(a.ux, a.uy, b.ux, b.uy);
}
__device__ __forceinline__ Dir2 shfl_up_dir(const Dir2& v, int o) {
  Dir2 r;
  r.lx = __shfl_up_sync(0xFFFFFFFFu, v.lx, o);
  r.ly = __shfl_up_sync(0xFFFFFFFFu, v.ly, o);
  r.ux = __shfl_up_sync(0xFFFFFFFFu, v.ux, o);
  r.uy = __shfl_up_sync(0xFFFFFFFFu, v.uy, o);
  return r;
}
// Inclusive warp scan under combine (earlier lanes first).
__device__ __forceinline__ Dir2 warp_scan_dir(Dir2 v) {
  const int lane = threadIdx.x & 31;
  #pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    Dir2 t = shfl_up_dir(v, o);
    if (lane >= o) { combine(t, v); v = t; }
  }
  return v;
}

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
  // The sort leaves its result in buffer a after an even number of passes.
  const bool in_b = (plan->npasses & 1u) != 0;
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

__device__ __forceinline__ bool last_block(Plan* plan, int ctr, bool* s_last) {
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) *s_last = atomicAdd(&plan->ctr[ctr], 1u) == gridDim.x - 1;
  __syncthreads();
  if (*s_last) __threadfence();
  return *s_last;
}

constexpr u64 kDirValid = 1ull << 63;
__device__ __forceinline__ u64 pack_dir(int dx, int dy) {
  return kDirValid | ((u64)(u32)(-dx) << 32) | (u64)(u32)(dy + (1 << 30));
}
__device__ __forceinline__ void unpack_dir(u64 w, int& dx, int& dy) {
  dx = -(int)((w >> 32) & 0x7FFFFFFFu);
  dy = (int)((long long)(u32)w - (1ll << 30));
}
__device__ __forceinline__ Dir2 shfl_xor_dir(const Dir2& v, int o) {
  Dir2 r;
  r.lx = __shfl_xor_sync(0xFFFFFFFFu, v.lx, o);
  r.ly = __shfl_xor_sync(0xFFFFFFFFu, v.ly, o);
  r.ux = __shfl_xor_sync(0xFFFFFFFFu, v.ux, o);
  r.uy = __shfl_xor_sync(0xFFFFFFFFu, v.uy, o);
  return r;
}

// Exclusive prefix of chunk c (one warp): lane l inspects chunk
// base - l for base = c - 1, c - 33, ...; in each region every chunk up to
// the nearest inclusive prefix contributes.  False (ERR_TIMEOUT set) if a
// predecessor published nothing within the spin limit.
__device__ __forceinline__ bool lookback_dir(K4Chunk* chunks, u32 c, Plan* plan, u32 spin,
                                             Dir2 ident, Dir2* out) {
  const int lane = threadIdx.x & 31;
  Dir2 acc = ident;
  bool done_lo = false, done_up = false;
  long long base = (long long)c - 1;
  while (base >= 0 && !(done_lo && done_up)) {
    const long long t = base - lane;
    // Before chunk 0 the identity acts as an inclusive prefix.
    u64 il = kDirValid, iu = kDirValid, al = 0, au = 0;
    bool bad = false;
    if (t >= 0) {
      K4Chunk* ch = &chunks[t];
      u32 it = 0;
      for (;;) {
        il = ld_relaxed_u64(&ch->inc_lo); iu = ld_relaxed_u64(&ch->inc_up);
        al = ld_relaxed_u64(&ch->agg_lo); au = ld_relaxed_u64(&ch->agg_up);
        if (((il | al) & kDirValid) && ((iu | au) & kDirValid)) break;
        if (++it > spin || aborted(plan)) { bad = true; break; }
        spin_pause(it);
      }
    }
    if (__any_sync(0xFFFFFFFFu, bad)) {
      if (lane == 0) flag_error(plan, ERR_TIMEOUT);
      return false;
    }
    Dir2 v = ident;
    const u32 ml = __ballot_sync(0xFFFFFFFFu, (il & kDirValid) != 0);
    const u32 mu = __ballot_sync(0xFFFFFFFFu, (iu & kDirValid) != 0);
    const int sl = ml ? (__ffs(ml) - 1) : 31, su = mu ? (__ffs(mu) - 1) : 31;
    if (t >= 0 && !done_lo && lane <= sl) unpack_dir((il & kDirValid) ? il : al, v.lx, v.ly);
    if (t >= 0 && !done_up && lane <= su) unpack_dir((iu & kDirValid) ? iu : au, v.ux, v.uy);
    #pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const Dir2 w = shfl_xor_dir(v, o);
      combine(v, w);
    }
    combine(acc, v);
    done_lo = done_lo || ml != 0u;
    done_up = done_up || mu != 0u;
    base -= 32;
  }
  *out = acc;
  return true;
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
  if (plan->error & ERR_RANGE) return;
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
    if (threadIdx.x == 0) chunks[c].cnt = make_uint2(tl, tu);
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
  const u32 per = (nchunks + K4_BLOCK - 1) / K4_BLOCK;
  const u32 lo = min(nchunks, threadIdx.x * per), hi = min(nchunks, lo + per);
  u32 sl = 0, su = 0;
  for (u32 c = lo; c < hi; ++c) {
    const volatile u32* q = reinterpret_cast<const volatile u32*>(&chunks[c].cnt);
    sl += q[0]; su += q[1];
  }
  u32 il = sl, iu = su;
  #pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const u32 t0 = __shfl_up_sync(0xFFFFFFFFu, il, o);
    const u32 t1 = __shfl_up_sync(0xFFFFFFFFu, iu, o);
    if (lane >= o) { il += t0; iu += t1; }
  }
  if (lane == 31) { s_wc[wid][0] = il; s_wc[wid][1] = iu; }
  __syncthreads();
  u32 ol = 0, ou = 0;
  for (int w = 0; w < wid; ++w) { ol += s_wc[w][0]; ou += s_wc[w][1]; }
  u32 rl = ol + il - sl, ru = ou + iu - su;
  for (u32 c = lo; c < hi; ++c) {
    const volatile u32* q = reinterpret_cast<const volatile u32*>(&chunks[c].cnt);
    const u32 a = q[0], b = q[1];
    chunks[c].off = make_uint2(rl, ru);
    rl += a; ru += b;
  }
  if (threadIdx.x == K4_BLOCK - 1) {
    const u32 r_lo = ol + il, r_up = ou + iu;
    plan->r_lo = r_lo;
    plan->r_up = r_up;
    const int i_a = plan->ext_idx[0], i_b = plan->ext_idx[1];
    lo_xy[0] = make_int2(g.ax, g.ay); lo_idx[0] = i_a;
    up_xy[0] = make_int2(g.ax, g.ay); up_idx[0] = i_a;
    if (r_lo + 1 < g.s + 2) { lo_xy[r_lo + 1] = make_int2(g.bx, g.by); lo_idx[r_lo + 1] = i_b; }
    if (r_up + 1 < g.s + 2) { up_xy[r_up + 1] = make_int2(g.bx, g.by); up_idx[r_up + 1] = i_b; }
  }
}

__global__ void __launch_bounds__(K4_BLOCK)
k4_compact(Plan* plan, const K4Chunk* __restrict__ chunks, const int2* __restrict__ t_lo_xy,
           const int* __restrict__ t_lo_idx, const int2* __restrict__ t_up_xy,
           const int* __restrict__ t_up_idx, int2* __restrict__ lo_xy, int* __restrict__ lo_idx,
           int2* __restrict__ up_xy, int* __restrict__ up_idx) {
  if (plan->error & (ERR_RANGE | ERR_TIMEOUT)) return;
  const u32 s = plan->s;
  const u32 nchunks = (s + K4_CHUNK - 1) / K4_CHUNK;
  for (u32 c = blockIdx.x; c < nchunks; c += gridDim.x) {
    const uint2 cnt = chunks[c].cnt, off = chunks[c].off;
    for (u32 j = threadIdx.x; j < cnt.x; j += K4_BLOCK) {
      const u32 d = 1 + off.x + j;
      if (d < s + 1) { lo_xy[d] = t_lo_xy[c * K4_CHUNK + j]; lo_idx[d] = t_lo_idx[c * K4_CHUNK + j]; }
      else flag_error(plan, ERR_INTERNAL);
    }
    for (u32 j = threadIdx.x; j < cnt.y; j += K4_BLOCK) {
      const u32 d = 1 + off.y + j;
      if (d < s + 1) { up_xy[d] = t_up_xy[c * K4_CHUNK + j]; up_idx[d] = t_up_idx[c * K4_CHUNK + j]; }
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
  k4_compact<<<grid, K4_BLOCK, 0, st>>>(plan, ch, t_lo_xy, t_lo_idx, t_up_xy, t_up_idx, lo_xy, lo_idx,
                                        up_xy, up_idx);
  return cudaGetLastError();
}

}  // namespace gbh
