// The second-round filter's scan state (Section 2.2, Figure 2, as an
// exclusive prefix max per region), shared by K4 (k4_regions.cu, over
// chunks of the sorted survivors) and the bucket sort (k3_bucket.cu, over
// its groups of bins): direction pairs, their combination, warp scans, the
// per-chunk look-back records and the decoupled look-back over them, and
// the last block's turn of the per-chunk kept counts into offsets.
#pragma once

#include "hull_internal.cuh"

namespace gbh {

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
  u32 base;               // first staging slot of the chunk's kept points
  u32 pad0;
  u64 pad1;
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
__device__ __forceinline__ Dir2 shfl_dir(const Dir2& v, int src) {
  Dir2 r;
  r.lx = __shfl_sync(0xFFFFFFFFu, v.lx, src);
  r.ly = __shfl_sync(0xFFFFFFFFu, v.ly, src);
  r.ux = __shfl_sync(0xFFFFFFFFu, v.ux, src);
  r.uy = __shfl_sync(0xFFFFFFFFu, v.uy, src);
  return r;
}
// Inclusive warp scan under combine (earlier lanes first); lanes below W
// see exactly the lanes before them, W a power of two <= 32.
template <int W = 32>
__device__ __forceinline__ Dir2 warp_scan_dir(Dir2 v) {
  const int lane = threadIdx.x & 31;
  #pragma unroll
  for (int o = 1; o < W; o <<= 1) {
    Dir2 t = shfl_up_dir(v, o);
    if (lane >= o) { combine(t, v); v = t; }
  }
  return v;
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

// Run by one whole block after every chunk published its kept counts:
// turns the counts of chunks [0, nrec) into exclusive offsets (per region),
// sets r_lo / r_up and writes P_0 and P_l at both ends of both region lists
// (capacity s + 2 each).  `red` is shared scratch of 2 * (blockDim.x / 32) words.
__device__ __forceinline__ void region_offsets(Plan* plan, K4Chunk* chunks, u32 nrec, u32 s, u32* red,
                                               int2* lo_xy, int* lo_idx, int2* up_xy, int* up_idx) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const u32 nt = blockDim.x;
  const u32 per = (nrec + nt - 1) / nt;
  const u32 lo = min(nrec, threadIdx.x * per), hi = min(nrec, lo + per);
  // The counts of a batch of records are loaded together (one round trip).
  constexpr int RB = 8;
  u32 sl = 0, su = 0;
  for (u32 cb = lo; cb < hi; cb += RB) {
    unsigned long long v[RB];
    #pragma unroll
    for (int q = 0; q < RB; ++q)
      v[q] = cb + q < hi ? *reinterpret_cast<const volatile unsigned long long*>(&chunks[cb + q].cnt) : 0ull;
    #pragma unroll
    for (int q = 0; q < RB; ++q) { sl += (u32)v[q]; su += (u32)(v[q] >> 32); }
  }
  u32 il = sl, iu = su;
  #pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const u32 t0 = __shfl_up_sync(0xFFFFFFFFu, il, o);
    const u32 t1 = __shfl_up_sync(0xFFFFFFFFu, iu, o);
    if (lane >= o) { il += t0; iu += t1; }
  }
  if (lane == 31) { red[2 * wid] = il; red[2 * wid + 1] = iu; }
  __syncthreads();
  u32 ol = 0, ou = 0;
  for (int w = 0; w < wid; ++w) { ol += red[2 * w]; ou += red[2 * w + 1]; }
  u32 rl = ol + il - sl, ru = ou + iu - su;
  for (u32 cb = lo; cb < hi; cb += RB) {
    unsigned long long v[RB];
    #pragma unroll
    for (int q = 0; q < RB; ++q)
      v[q] = cb + q < hi ? *reinterpret_cast<const volatile unsigned long long*>(&chunks[cb + q].cnt) : 0ull;
    #pragma unroll
    for (int q = 0; q < RB; ++q) {
      if (cb + q < hi) chunks[cb + q].off = make_uint2(rl, ru);
      rl += (u32)v[q];
      ru += (u32)(v[q] >> 32);
    }
  }
  if (threadIdx.x == nt - 1) {
    const u32 r_lo = ol + il, r_up = ou + iu;
    plan->r_lo = r_lo;
    plan->r_up = r_up;
    const int i_a = plan->ext_idx[0], i_b = plan->ext_idx[1];
    const int ax = plan->ext_x[0], ay = plan->ext_y[0], bx = plan->ext_x[1], by = plan->ext_y[1];
    lo_xy[0] = make_int2(ax, ay); lo_idx[0] = i_a;
    up_xy[0] = make_int2(ax, ay); up_idx[0] = i_a;
    if (r_lo + 1 < s + 2) { lo_xy[r_lo + 1] = make_int2(bx, by); lo_idx[r_lo + 1] = i_b; }
    if (r_up + 1 < s + 2) { up_xy[r_up + 1] = make_int2(bx, by); up_idx[r_up + 1] = i_b; }
  }
}

}  // namespace gbh
