// K3 of the hull pipeline: bucket sort of the filter's survivors (Section
// 2.1 step 4, Section 3.3), ascending by (key, index): the order of a stable
// sort by key of the survivors in index order, which is the order the
// paper's sort_by_key gives; the key is the lexicographic (x, y) key.
//
// The pipeline's sort moves the survivors' pairs twice after the filter
// instead of once per radix digit:
//   1. the fused filter (k2_fused.cu) adds every survivor to its bin's total
//      (a bin = the top kBinBits of the key) and writes its (key, index)
//      pair in any order; its last block turns the totals into bin starts
//      and groups of consecutive bins (bins.cuh), and k2_place moves every
//      pair into its coarse bin (kFinePerCoarse consecutive bins);
//   2. k3_split spreads every coarse bin over its bins (with the tiles'
//      direction aggregates, from which k_bin_prefix scans every bin's
//      second-round prefix), and k3_bucket takes one group at a time into
//      shared memory: a counting pass over kSubBins sub-bins of the group's
//      exact key range, then either Figure 2 on the binned group (each
//      thread owns whole sub-bins and orders only its candidates) or, for
//      the stage entry point and crowded groups, the order inside every
//      sub-bin by rank counting (a bitonic network when a sub-bin is
//      crowded).
// The radix-pass path (hull_stage_bucket_sort, the array sort) bins an
// index-ordered survivor array itself (launch_array_bins).
//
// Groups: bin b starts a new group when floor(start_b / T) differs from
// its predecessor's (T = kGroupTarget), when it or its predecessor holds
// more than T survivors, or when b starts a coarse bin (kFinePerCoarse
// consecutive bins).  A group of small bins then starts and ends inside
// one window of T positions plus its last bin, so it holds fewer than 2T =
// kGroupCap survivors; a larger bin is a group of its own.  Since a group
// spans at most kFinePerCoarse bins, each bin's key range takes at least
// kSubBins / kFinePerCoarse sub-bins of the group's map, so a bin of up to
// T points spread over its range cannot crowd them (one dense bin in a
// group of many sparse ones used to send the whole group to the bitonic
// network).  A bin above
// kGroupCap is split once more through global memory by its next kSubBits
// key bits; if one of those sub-bins is still above kGroupCap (heavy
// duplication, or a few points spread over a huge bounding box) the block
// sets ERR_FALLBACK and the host reruns the call on the radix passes of
// k3_sort.cu.
#include <cstddef>

#include "hull_internal.cuh"
#include "kernels.h"
#include "bins.cuh"
#include "regions.cuh"

#ifdef GBH_DEBUG_CHECKS
#include <cstdio>
#endif

namespace gbh {

namespace {

#ifndef GBH_KB_BLOCK
#define GBH_KB_BLOCK 512
#endif
constexpr int KB_BLOCK = GBH_KB_BLOCK;
constexpr int KB_MIN_BLOCKS = 2;                    // two blocks per SM (the shared-memory arrays)
constexpr int KB_WARPS = KB_BLOCK / 32;
constexpr int KB_ITEMS = kGroupCap / KB_BLOCK;     // keys per thread in a full group
constexpr int KB_HALF = KB_ITEMS / 2;              // keys loaded per batch
static_assert(KB_HALF * 2 == KB_ITEMS, "two load batches");
constexpr u32 kCrowded = 32;                       // largest sub-bin ordered by rank counting
constexpr u32 kBinnedMax = 32;                     // most pairs a thread scans unsorted (one mask bit each)
constexpr int KB_SCAN_PER = (kSubBins) / KB_BLOCK; // sub-bin counters per thread in the scan
static_assert(KB_SCAN_PER * KB_BLOCK == kSubBins, "whole counters per thread");
static_assert(kGroupCap <= (1 << 13) && kSubBits <= 19, "rank and sub-bin packed in 32 bits");
constexpr int kScratchWords = kSubBins + 1 + kSubBins / 32;   // per block: split starts, piece flags

struct BucketSmem {
  u64 key[kGroupCap];      // sorted pairs, slot phys(i) for position i
  u32 val[kGroupCap];
  u32 cnt[kSubBins + 1];
  u32 wsum[KB_WARPS];
  u32 misc[8];             // [0] big-bin piece end, [1] claimed group, [2..4] sub-bin map
  // second round
  Dir2 dirs[KB_WARPS];     // per-warp direction aggregates (each includes the piece's prefix)
  Dir2 wtot;               // prefix through the whole piece
  Dir2 carry;              // prefix through the group's positions scanned so far
  u32 kwl[KB_WARPS][2];    // per-warp kept counts (lower, upper)
  u32 kept[2];             // the group's kept points so far
  // the next group, fetched while the current one is processed
  __align__(16) u64 ninc[2];   // its exclusive prefix words (lower, upper)
  uint2 nab[2];            // groups[id], groups[id + 1]
  u32 nid;                 // its id (>= the group count: none)
  u32 nerr;                // the plan's error word, fetched with it
};

// Shared-memory slot of sorted position i: the low five bits are XORed
// with the next five, so that threads reading consecutive runs of 8 or 16
// positions hit different banks (a bijection inside every 32 slots).
__device__ __forceinline__ u32 phys(u32 i) { return i ^ ((i >> 5) & 31u); }

#ifdef GBH_DEBUG_CHECKS
__device__ unsigned int g_dbg_reported = 0;
#define DBG_REPORT(code, a, b, c, d)                                                                   \
  do {                                                                                                  \
    if (atomicCAS(&g_dbg_reported, 0u, 1u) == 0u)                                                       \
      printf("GBH_DEBUG k3 check %d failed: block %d thread %d: %llu %llu %llu %llu\n", (int)(code),    \
             (int)blockIdx.x, (int)threadIdx.x, (unsigned long long)(a), (unsigned long long)(b),      \
             (unsigned long long)(c), (unsigned long long)(d));                                        \
  } while (0)
#endif

__device__ __forceinline__ u32 ceil_log2(u32 v) { return v <= 1u ? 0u : 32u - __clz(v - 1u); }

__device__ __forceinline__ bool pair_less(u64 ka, u32 va, u64 kb, u32 vb) {
  return ka < kb || (ka == kb && va < vb);
}

// Sum of the values of warps [0, wid): every lane passes warp `lane`'s
// value (lanes >= KB_WARPS pass anything); a scan across the lanes.
__device__ __forceinline__ u32 warps_before(u32 x, int wid) {
  const int lane = threadIdx.x & 31;
  if (lane >= KB_WARPS) x = 0u;
  #pragma unroll
  for (int o = 1; o < KB_WARPS; o <<= 1) {
    const u32 t = __shfl_up_sync(0xFFFFFFFFu, x, o);
    if (lane >= o) x += t;
  }
  const u32 b = __shfl_sync(0xFFFFFFFFu, x, wid > 0 ? wid - 1 : 0);
  return wid > 0 ? b : 0u;
}

// Exclusive scan of S.cnt[0..kSubBins) in place, S.cnt[kSubBins] = total.
// Returns (on every thread) kCrowdedFlag when some counter exceeds kCrowded
// and kHeavyFlag when the KB_SCAN_PER counters of some thread sum to more
// than kBinnedMax (a crowded sub-bin makes its thread heavy too).
constexpr int kCrowdedFlag = 1, kHeavyFlag = 2;
__device__ __forceinline__ int scan_counts(BucketSmem& S) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  static_assert(KB_SCAN_PER == 8, "two 16-byte words of counters per thread");
  u32 v[KB_SCAN_PER];
  {
    const uint4 c0 = *reinterpret_cast<const uint4*>(&S.cnt[threadIdx.x * KB_SCAN_PER]);
    const uint4 c1 = *reinterpret_cast<const uint4*>(&S.cnt[threadIdx.x * KB_SCAN_PER + 4]);
    v[0] = c0.x; v[1] = c0.y; v[2] = c0.z; v[3] = c0.w; v[4] = c1.x; v[5] = c1.y; v[6] = c1.z; v[7] = c1.w;
  }
  u32 sum = 0, mx = 0;
  #pragma unroll
  for (int j = 0; j < KB_SCAN_PER; ++j) {
    sum += v[j];
    mx = max(mx, v[j]);
  }
  u32 inc = sum;
  #pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const u32 t = __shfl_up_sync(0xFFFFFFFFu, inc, o);
    if (lane >= o) inc += t;
  }
  if (lane == 31) S.wsum[wid] = inc;
  const int flags = (mx > kCrowded ? kCrowdedFlag : 0) | (sum > kBinnedMax ? kHeavyFlag : 0);
  int st = __syncthreads_or(flags) != 0 ? kHeavyFlag : 0;
  if (st) st |= __syncthreads_or(flags & kCrowdedFlag) != 0 ? kCrowdedFlag : 0;
  u32 run = inc - sum + warps_before(S.wsum[lane < KB_WARPS ? lane : 0], wid);
  u32 r[KB_SCAN_PER];
  #pragma unroll
  for (int j = 0; j < KB_SCAN_PER; ++j) {
    r[j] = run;
    run += v[j];
  }
  *reinterpret_cast<uint4*>(&S.cnt[threadIdx.x * KB_SCAN_PER]) = make_uint4(r[0], r[1], r[2], r[3]);
  *reinterpret_cast<uint4*>(&S.cnt[threadIdx.x * KB_SCAN_PER + 4]) = make_uint4(r[4], r[5], r[6], r[7]);
  if (threadIdx.x == KB_BLOCK - 1) S.cnt[kSubBins] = run;
  __syncthreads();
  return st;
}

// Bitonic network over S.key/S.val[0, m), padded to a power of two with
// pairs above every real one ((key, value) pairs are distinct, so any
// correct sort gives the same order).
__device__ void bitonic(BucketSmem& S, u32 m) {
  u32 P = 1;
  while (P < m) P <<= 1;
  for (u32 i = m + threadIdx.x; i < P; i += KB_BLOCK) {
    S.key[phys(i)] = ~0ull;
    S.val[phys(i)] = ~0u;
  }
  __syncthreads();
  for (u32 k = 2; k <= P; k <<= 1) {
    for (u32 j = k >> 1; j > 0; j >>= 1) {
      for (u32 i = threadIdx.x; i < P; i += KB_BLOCK) {
        const u32 l = i ^ j;
        if (l > i) {
          const u32 pi = phys(i), pl = phys(l);
          const u64 ki = S.key[pi], kl = S.key[pl];
          const u32 vi = S.val[pi], vl = S.val[pl];
          const bool up = (i & k) == 0;
          const bool swap = up ? pair_less(kl, vl, ki, vi) : pair_less(ki, vi, kl, vl);
          if (swap) {
            S.key[pi] = kl; S.key[pl] = ki;
            S.val[pi] = vl; S.val[pl] = vi;
          }
        }
      }
      __syncthreads();
    }
  }
}

// Source loads: through the read-only path when the source is not written
// during the kernel (RO), else plain coherent loads.
template <bool RO, typename T>
__device__ __forceinline__ T load_src(const T* p) {
  if (RO) return __ldg(p);
  return *p;
}

// Sub-bin of a key offset in [0, top]: the offset cut or widened to
// exactly 32 significant bits (x), then the high word of x * M, where
// M is at most kSubBins 2^32 / (largest x + 1).  Monotone in the offset, it
// spreads the whole range evenly over the kSubBins sub-bins (a shift by a
// power of two would leave up to half of them empty and crowd the rest).
struct SubMap {
  u32 esh, lsh, M;
};

__device__ __forceinline__ SubMap make_submap(u64 top) {
  SubMap f;
  const u32 kb = top ? 64u - (u32)__clzll((long long)top) : 0u;
  f.esh = kb > 32u ? kb - 32u : 0u;
  f.lsh = (kb > 0u && kb < 32u) ? 32u - kb : 0u;
  // M <= kSubBins 2^32 / (xmax + 1) from the top 12 bits of xmax (which is
  // in [2^31, 2^32) when kb > 0): y 2^20 > xmax, within 1/2048 of it.
  const u32 y = (u32)(((top >> f.esh) << f.lsh) >> 20) + 1u;
  f.M = kb ? ((u32)kSubBins << 12) / y : 0u;
  return f;
}

// Largest offset of nb >= 1 consecutive units of 2^sh keys (2^64 - 1 at most).
__device__ __forceinline__ u64 span_top(u32 nb, u32 sh) {
  return ((u64)(nb - 1u) << sh) + ((1ull << sh) - 1ull);
}

__device__ __forceinline__ u32 sub_of(const SubMap& f, u64 off) {
  return __umulhi((u32)(off >> f.esh) << f.lsh, f.M);
}

// ---- the second round, fused (Section 2.2, Figure 2): geometry of the
// split line P_0 -> P_l and of the directions d(p) = p - P_l.
struct RG {
  int x0, y0, ax, ay, bx, by, ux, uy;
  int dx0, dy0;           // key origin minus P_l
  u32 ybits;
  u64 ymask;
  Dir2 ident;
};

__device__ __forceinline__ RG make_rg(const Plan* plan) {
  RG g;
  g.x0 = plan->key_x0; g.y0 = plan->key_y0;
  g.ybits = plan->ybits;
  g.ymask = g.ybits ? ((~0ull) >> (64 - g.ybits)) : 0ull;
  g.ax = plan->ext_x[0]; g.ay = plan->ext_y[0];     // P_0 = P_minx
  g.bx = plan->ext_x[1]; g.by = plan->ext_y[1];     // P_l = P_maxx
  g.ux = g.bx - g.ax; g.uy = g.by - g.ay;
  g.dx0 = g.x0 - g.bx; g.dy0 = g.y0 - g.by;
  g.ident = {g.ax - g.bx, g.ay - g.by, g.ax - g.bx, g.ay - g.by};
  return g;
}

// Point of a key, and its region: -1 lower (right of P_0 -> P_l), +1 upper, 0 on the line.
__device__ __forceinline__ int decode_side(const RG& g, u64 k, int& px, int& py) {
  px = g.x0 + (int)(u32)(k >> g.ybits);
  py = g.y0 + (int)(u32)(k & g.ymask);
  const long long o = cross2(g.ux, g.uy, px - g.ax, py - g.ay);
  return o < 0 ? -1 : (o > 0 ? 1 : 0);
}

// Direction d = p - P_l of a key's point, and its region: the sign of
// cross(P_l - P_0, d), which equals cross(P_l - P_0, p - P_0) (the same
// value as decode_side's, without decoding p).
__device__ __forceinline__ long long key_dir(const RG& g, u64 k, int& vx, int& vy) {
  vx = (int)(u32)(k >> g.ybits) + g.dx0;
  vy = (int)(u32)(k & g.ymask) + g.dy0;
  return cross2(g.ux, g.uy, vx, vy);
}

__device__ __forceinline__ void add_dir(Dir2& a, const RG& g, u64 k) {
  int vx, vy;
  const long long o = key_dir(g, k, vx, vy);
  if (o < 0) cmax(a.lx, a.ly, vx, vy);
  else if (o > 0) cmin(a.ux, a.uy, vx, vy);
}


// A direction pair (lower, upper words; a word without its valid bit is
// the identity's).
__device__ __forceinline__ Dir2 unpack_pair(u64 wl, u64 wu, const RG& rg) {
  Dir2 v = rg.ident;
  if (wl & kDirValid) unpack_dir(wl, v.lx, v.ly);
  if (wu & kDirValid) unpack_dir(wu, v.ux, v.uy);
  return v;
}

// The second round run by the pipeline's sort: every group's record holds
// its exclusive prefix (k_bin_prefix) and receives its kept
// counts; kept points are staged in t_* and the last block turns the counts
// into offsets and fills both ends of the region lists.
struct Fused {
  K4Chunk* recs;
  int2* t_lo_xy; int* t_lo_idx; int2* t_up_xy; int* t_up_idx;
  int2* lo_xy; int* lo_idx; int2* up_xy; int* up_idx;
  const u64* bpre;         // every bin's exclusive prefix (k_bin_prefix)
};

// The second round's early drop (the fused path): a pair whose point lies
// within the prefix extreme of all points in earlier bins cannot be kept
// (it does not change the running extreme either), so the sort skips it.
// bpre == nullptr: no drop.  The group's first nb <= KB_WARPS prefixes are
// cached in S.dirs (free until the second round).
struct Drop {
  const u64* bpre;
  u32 bin0, nb, fshift;
};

// Next position to visit among the bits of `mask` (bit j: position p0 + j),
// in (key, value) order.  Sorted pairs: the lowest bit.  Binned pairs (a
// thread's positions are whole sub-bins, in sub-bin order, each in any
// order inside): the smallest (key, value) among the bits that share the
// lowest bit's sub-bin.
__device__ __forceinline__ u32 next_visit(const BucketSmem& S, u32 mask, u32 p0, bool binned, const SubMap& f,
                                          u64 klo) {
  const u32 j0 = __ffs(mask) - 1;
  u32 rest = mask & (mask - 1u);
  if (!binned || !rest) return j0;
  u64 bk = S.key[phys(p0 + j0)];
  u32 bv = S.val[phys(p0 + j0)];
  const u32 e = S.cnt[sub_of(f, bk - klo) + 1] - p0;   // end of that sub-bin, at most 32
  if (e < 32u) rest &= (1u << e) - 1u;
  u32 best = j0;
  for (; rest; rest &= rest - 1u) {
    const u32 j = __ffs(rest) - 1;
    const u64 kj = S.key[phys(p0 + j)];
    const u32 vj = S.val[phys(p0 + j)];
    if (pair_less(kj, vj, bk, bv)) { best = j; bk = kj; bv = vj; }
  }
  return best;
}

// Figure 2 over the m pairs in shared memory, starting from the prefix
// S.carry: keeps a point when its direction is strictly beyond the running
// extreme of its region, stages the kept points from slot
// `slot0 + S.kept[region]` and advances S.carry and S.kept.  Sorted pairs:
// thread t takes positions [t R, t R + R).  Binned pairs (sorted by
// sub-bin only; klo and the sub-bin map of sort_into_smem give each key's
// sub-bin): thread t takes its KB_SCAN_PER sub-bins, whole.
//
// One pass per thread keeps loc = the extreme of S.carry and its positions
// so far, and marks as candidates the positions strictly beyond lsb, the
// extreme through the sub-bins before the position's own (sorted pairs:
// every position is a sub-bin, lsb = loc).  A position that is not a
// candidate lies within lsb, i.e. within the directions of points before
// it in the true order, and is dropped whatever the order inside its
// sub-bin.  So the true running extreme before a position is the thread's
// exclusive prefix E combined with the candidates before it, and the
// second pass visits the candidates only, each sub-bin's in (key, value)
// order.  The scan across threads combines the loc values (S.carry is
// idempotent under the combination, so that is E).
__device__ void scan_piece(BucketSmem& S, const Fused& F, u32 m, u32 slot0, u32 s, const RG& rg, Plan* plan,
                           bool binned, u64 klo) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const SubMap f = {S.misc[2], S.misc[3], S.misc[4]};
  u32 p0, p1;
  if (binned) {
    p0 = S.cnt[threadIdx.x * KB_SCAN_PER];
    p1 = S.cnt[threadIdx.x * KB_SCAN_PER + KB_SCAN_PER];
  } else {
    const u32 R = (m + KB_BLOCK - 1) / KB_BLOCK;
    p0 = min(m, threadIdx.x * R);
    p1 = min(m, p0 + R);
  }
  // Bit j of smask: position p0 + j starts a sub-bin (sorted pairs: every
  // position does).
  u32 smask = 0xFFFFFFFFu;
  if (binned) {
    const uint4 c0 = *reinterpret_cast<const uint4*>(&S.cnt[threadIdx.x * KB_SCAN_PER]);
    const uint4 c1 = *reinterpret_cast<const uint4*>(&S.cnt[threadIdx.x * KB_SCAN_PER + 4]);
    const u32 st[KB_SCAN_PER] = {c0.x, c0.y, c0.z, c0.w, c1.x, c1.y, c1.z, c1.w};
    smask = 0u;
    #pragma unroll
    for (int j = 0; j < KB_SCAN_PER; ++j)
      if (st[j] < p1) smask |= 1u << (st[j] - p0);
  }
  const Dir2 carry = S.carry;
  Dir2 loc = carry, lsb = carry;
  u32 cand = 0;                                   // bit j: position p0 + j is a candidate
  for (u32 pb = p0; pb < p1; pb += 4) {
    u64 kq[4];                                    // four keys loaded together
    #pragma unroll
    for (int q = 0; q < 4; ++q) kq[q] = pb + q < p1 ? S.key[phys(pb + q)] : 0ull;
    #pragma unroll
    for (int q = 0; q < 4; ++q) {
      const u32 j = pb + q - p0;
      if (pb + q >= p1) break;
      if ((smask >> j) & 1u) lsb = loc;
      int vx, vy;
      const long long o = key_dir(rg, kq[q], vx, vy);
      if (o < 0) {
        if (cross2(lsb.lx, lsb.ly, vx, vy) > 0) {
          cand |= 1u << j;
          if (cross2(loc.lx, loc.ly, vx, vy) > 0) { loc.lx = vx; loc.ly = vy; }
        }
      } else if (o > 0) {
        if (cross2(lsb.ux, lsb.uy, vx, vy) < 0) {
          cand |= 1u << j;
          if (cross2(loc.ux, loc.uy, vx, vy) < 0) { loc.ux = vx; loc.uy = vy; }
        }
      }
    }
  }
  // Exclusive prefix of this thread: warp scan, then the warps' totals.
  const Dir2 inc = warp_scan_dir(loc);
  const Dir2 lex = shfl_up_dir(inc, 1);
  if (lane == 31) S.dirs[wid] = inc;
  __syncthreads();
  // Every warp scans the warps' aggregates itself (each includes S.carry,
  // which the combination absorbs, so lanes past the warps may pass it).
  const Dir2 wi = warp_scan_dir<KB_WARPS>(lane < KB_WARPS ? S.dirs[lane] : carry);
  Dir2 ex = shfl_dir(wi, wid > 0 ? wid - 1 : 0);
  if (wid == 0) ex = carry;
  if (wid == 0 && lane == KB_WARPS - 1) S.wtot = wi;
  if (lane > 0) combine(ex, lex);
  // Second pass: the candidates only, in (key, value) order.
  u32 keep_lo = 0, keep_up = 0;
  Dir2 prev = ex;                                 // E combined with the candidates visited so far
  for (u32 c = cand; c;) {
    const u32 j = next_visit(S, c, p0, binned, f, klo);
    c &= ~(1u << j);
    int px, py;
    const int sd = decode_side(rg, S.key[phys(p0 + j)], px, py);
    const int vx = px - rg.bx, vy = py - rg.by;
    if (sd < 0) {
      if (cross2(prev.lx, prev.ly, vx, vy) > 0) { keep_lo |= 1u << j; prev.lx = vx; prev.ly = vy; }
    } else {
      if (cross2(prev.ux, prev.uy, vx, vy) < 0) { keep_up |= 1u << j; prev.ux = vx; prev.uy = vy; }
    }
  }
  const u32 c_lo = __popc(keep_lo), c_up = __popc(keep_up);
  u32 i_lo = c_lo, i_up = c_up;
  #pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const u32 t0 = __shfl_up_sync(0xFFFFFFFFu, i_lo, o);
    const u32 t1 = __shfl_up_sync(0xFFFFFFFFu, i_up, o);
    if (lane >= o) { i_lo += t0; i_up += t1; }
  }
  if (lane == 31) { S.kwl[wid][0] = i_lo; S.kwl[wid][1] = i_up; }
  __syncthreads();
  const int wl_src = lane < KB_WARPS ? lane : 0;
  const u32 wl = warps_before(S.kwl[wl_src][0], wid), wu = warps_before(S.kwl[wl_src][1], wid);
  const u32 tl = warps_before(S.kwl[wl_src][0], KB_WARPS), tu = warps_before(S.kwl[wl_src][1], KB_WARPS);
  u32 pl = slot0 + S.kept[0] + wl + i_lo - c_lo;
  u32 pu = slot0 + S.kept[1] + wu + i_up - c_up;
  for (u32 c = keep_lo | keep_up; c;) {
    const u32 j = next_visit(S, c, p0, binned, f, klo);
    c &= ~(1u << j);
    int px, py;
    decode_side(rg, S.key[phys(p0 + j)], px, py);
    const int idx = (int)S.val[phys(p0 + j)];
    if (keep_lo & (1u << j)) {
      if (pl < s) { F.t_lo_xy[pl] = make_int2(px, py); F.t_lo_idx[pl] = idx; } else flag_error(plan, ERR_INTERNAL);
      ++pl;
    } else {
      if (pu < s) { F.t_up_xy[pu] = make_int2(px, py); F.t_up_idx[pu] = idx; } else flag_error(plan, ERR_INTERNAL);
      ++pu;
    }
  }
  // The piece's prefix for the next piece of the same group, and the kept counts.
  __syncthreads();
  if (threadIdx.x == 0) {
    S.carry = S.wtot;
    S.kept[0] += tl;
    S.kept[1] += tu;
  }
  __syncthreads();
}

// Starts group g's second round from its exclusive prefix (one thread).
__device__ __forceinline__ void start_group(BucketSmem& S) {
  Dir2 e;
  unpack_dir(S.ninc[0], e.lx, e.ly);
  unpack_dir(S.ninc[1], e.ux, e.uy);
  S.carry = e;
  S.kept[0] = S.kept[1] = 0u;
}

// Thread 0: starts the asynchronous fetch of group g's descriptor (its
// first position and bin, the next group's, and with DECIDE its prefix)
// into S.nab / S.ninc, with the plan's error word (a block stops claiming
// once a group needs the radix passes; nothing depends on seeing it at
// once), and records g in S.nid.
template <bool DECIDE>
__device__ __forceinline__ void fetch_group(BucketSmem& S, const Fused& F, const uint2* groups, u32 g, u32 ng,
                                            const Plan* plan) {
  S.nid = g;
  if (g >= ng) return;
  cp_async4(&S.nerr, &plan->error);
  cp_async8(&S.nab[0], &groups[g]);
  cp_async8(&S.nab[1], &groups[g + 1]);
  if (DECIDE) cp_async16(&S.ninc[0], &F.recs[g].inc_lo);
  cp_async_commit();
}


// Sorts the m <= kGroupCap pairs at [base, base + m) of (sk, sv), whose keys
// lie in [klo, klo + ktop], into shared memory (position i in slot
// phys(i)), ordered by (key, value).  Every thread of the block calls it.
// With allow_binned, when no thread's KB_SCAN_PER sub-bins hold more than
// kBinnedMax pairs, it stops once the pairs are in sub-bin order and
// returns true (binned: the pairs of a sub-bin in any order).
template <bool RO>
__device__ bool sort_into_smem(BucketSmem& S, const u64* sk, const u32* sv, u32 base, u32 m, u64 klo,
                               u64 ktop, Plan* plan, bool allow_binned, const Drop& dr, const RG& rg) {
  if (threadIdx.x == 0) {
    const SubMap f = make_submap(ktop);
    S.misc[2] = f.esh; S.misc[3] = f.lsh; S.misc[4] = f.M;
  }
  if (dr.bpre && threadIdx.x < min(dr.nb, (u32)KB_WARPS)) {
    const u32 q = dr.bin0 + threadIdx.x;
    S.dirs[threadIdx.x] = unpack_pair(__ldg(&dr.bpre[2 * q]), __ldg(&dr.bpre[2 * q + 1]), rg);
  }
  for (u32 i = threadIdx.x; i < (u32)kSubBins / 4; i += KB_BLOCK)
    reinterpret_cast<uint4*>(S.cnt)[i] = make_uint4(0u, 0u, 0u, 0u);
  if (threadIdx.x == 0) S.cnt[kSubBins] = 0u;
  __syncthreads();
  const SubMap f = {S.misc[2], S.misc[3], S.misc[4]};
  // Rank: every key's sub-bin and its arrival rank there.  The keys of a
  // batch are loaded before any of them is counted, so that the loads are
  // in flight together.
  u32 pk[KB_ITEMS];
  #pragma unroll
  for (int h = 0; h < 2; ++h) {
    #pragma unroll
    for (int q = 0; q < KB_HALF; ++q) pk[h * KB_HALF + q] = 0xFFFFFFFFu;
    if (h > 0 && m <= (u32)(KB_HALF * KB_BLOCK)) continue;
    u64 kk[KB_HALF];
    #pragma unroll
    for (int q = 0; q < KB_HALF; ++q) {
      const u32 i = (h * KB_HALF + q) * KB_BLOCK + threadIdx.x;
      kk[q] = i < m ? load_src<RO>(sk + base + i) : 0ull;
    }
    #pragma unroll
    for (int q = 0; q < KB_HALF; ++q) {
      const u32 i = (h * KB_HALF + q) * KB_BLOCK + threadIdx.x;
      if (i < m) {
        const u64 off = kk[q] - klo;
        if (off <= ktop) {
          bool keep = true;
          if (dr.bpre) {
            const u32 bi = (u32)(kk[q] >> dr.fshift) - dr.bin0;
            const Dir2 e = bi < (u32)KB_WARPS ? S.dirs[bi]
                                              : unpack_pair(__ldg(&dr.bpre[2 * (dr.bin0 + bi)]),
                                                            __ldg(&dr.bpre[2 * (dr.bin0 + bi) + 1]), rg);
            int vx, vy;
            const long long o = key_dir(rg, kk[q], vx, vy);
            keep = o < 0 ? cross2(e.lx, e.ly, vx, vy) > 0 : (o > 0 && cross2(e.ux, e.uy, vx, vy) < 0);
          }
          if (keep) {
            const u32 d = sub_of(f, off);
            pk[h * KB_HALF + q] = (d << 13) | atomicAdd(&S.cnt[d], 1u);
          }
        } else {
          flag_error(plan, ERR_INTERNAL);
        }
      }
    }
  }
  const int st = scan_counts(S);
#ifdef GBH_DEBUG_CHECKS
  if (S.cnt[kSubBins] != m) {
    if (threadIdx.x == 0) DBG_REPORT(2, base, m, S.cnt[kSubBins], ktop);
    flag_error(plan, ERR_INTERNAL);
  }
#endif
  // Place: the pairs of a batch are loaded together, then stored (the last
  // read of a read-only source: evict-first).
  const u64 pol_last = policy_evict_first();
  #pragma unroll
  for (int h = 0; h < 2; ++h) {
    if (h > 0 && m <= (u32)(KB_HALF * KB_BLOCK)) continue;
    u64 kk[KB_HALF];
    u32 vv[KB_HALF];
    #pragma unroll
    for (int q = 0; q < KB_HALF; ++q) {
      const u32 i = (h * KB_HALF + q) * KB_BLOCK + threadIdx.x;
      kk[q] = 0ull;
      vv[q] = 0u;
      if (i < m) {
        kk[q] = RO ? ld_hint_u64(sk + base + i, pol_last) : sk[base + i];
        vv[q] = RO ? ld_hint_u32(sv + base + i, pol_last) : sv[base + i];
      }
    }
    #pragma unroll
    for (int q = 0; q < KB_HALF; ++q) {
      const u32 t = pk[h * KB_HALF + q];
      if (t != 0xFFFFFFFFu) {
        const u32 p = phys(S.cnt[t >> 13] + (t & 8191u));
        S.key[p] = kk[q];
        S.val[p] = vv[q];
      }
    }
  }
  __syncthreads();
  if (allow_binned && !(st & kHeavyFlag)) return true;
  if (!(st & kCrowdedFlag)) {
    // Order every sub-bin by (key, value): each pair of a sub-bin of two or
    // more counts the pairs of its sub-bin below it (its rank there); after
    // a barrier the pairs not yet at their rank move there, reloaded from
    // the source.
    #pragma unroll
    for (int it = 0; it < KB_ITEMS; ++it) {
      const u32 t = pk[it];
      u32 np = 0xFFFFFFFFu;
      if (t != 0xFFFFFFFFu) {
        const u32 d = t >> 13, rk = t & 8191u;
        const u32 a = S.cnt[d], c = S.cnt[d + 1] - a;
        if (c > 1u) {
          const u32 ps = phys(a + rk);
          const u64 k = S.key[ps];
          const u32 v = S.val[ps];
          u32 r = 0;
          for (u32 j = 0; j < c; ++j) {
            const u32 q = phys(a + j);
            r += pair_less(S.key[q], S.val[q], k, v) ? 1u : 0u;
          }
          if (r != rk) np = a + r;
        }
      }
      pk[it] = np;
    }
    __syncthreads();
    #pragma unroll
    for (int h = 0; h < 2; ++h) {
      if (h > 0 && m <= (u32)(KB_HALF * KB_BLOCK)) continue;
      u64 kk[KB_HALF];
      u32 vv[KB_HALF];
      #pragma unroll
      for (int q = 0; q < KB_HALF; ++q) {
        const u32 i = (h * KB_HALF + q) * KB_BLOCK + threadIdx.x;
        kk[q] = 0ull;
        vv[q] = 0u;
        if (pk[h * KB_HALF + q] != 0xFFFFFFFFu) {
          kk[q] = load_src<RO>(sk + base + i);
          vv[q] = load_src<RO>(sv + base + i);
        }
      }
      #pragma unroll
      for (int q = 0; q < KB_HALF; ++q) {
        const u32 f = pk[h * KB_HALF + q];
        if (f != 0xFFFFFFFFu) {
          S.key[phys(f)] = kk[q];
          S.val[phys(f)] = vv[q];
        }
      }
    }
  } else {
    bitonic(S, S.cnt[kSubBins]);
  }
  __syncthreads();
  return false;
}

__device__ __forceinline__ void write_out(BucketSmem& S, u64* dk, u32* dv, u32 base, u32 m) {
  for (u32 i = threadIdx.x; i < m; i += KB_BLOCK) {
    dk[base + i] = S.key[phys(i)];
    dv[base + i] = S.val[phys(i)];
  }
  __syncthreads();
}

// A bin of m > kGroupCap pairs at [base, base + m) of (ak, av), keys in
// [klo, klo + 2^span): split by the next kSubBits key bits into (bk, bv),
// then sort the pieces of consecutive sub-bins in place there (DECIDE: run
// the second round over each sorted piece in order instead of writing it
// back).  `scratch` holds this block's sub-bin starts and piece flags.
template <bool DECIDE>
__device__ void big_bin(BucketSmem& S, const u64* __restrict__ ak, const u32* __restrict__ av,
                        u64* bk, u32* bv, u32 base, u32 m, u64 klo, u32 span, u32* scratch,
                        Plan* plan, const RG& rg, const Fused& F, u32 g) {
  const u32 sh = span > (u32)kSubBits ? span - (u32)kSubBits : 0u;
  u32* gstart = scratch;                     // kSubBins + 1
  u32* gflag = scratch + kSubBins + 1;       // kSubBins / 32 words
  for (u32 i = threadIdx.x; i <= (u32)kSubBins; i += KB_BLOCK) S.cnt[i] = 0u;
  __syncthreads();
  for (u32 i = threadIdx.x; i < m; i += KB_BLOCK) {
    const u64 k = ak[base + i];
    const u64 d64 = (k - klo) >> sh;
    if (d64 < (u64)kSubBins) atomicAdd(&S.cnt[(u32)d64], 1u);
    else flag_error(plan, ERR_INTERNAL);
  }
  scan_counts(S);
  // Piece flags (the group rule again, over sub-bins) and the starts.
  const u32 T = (u32)kGroupTarget;
  for (u32 d0 = 0; d0 < (u32)kSubBins; d0 += KB_BLOCK) {
    const u32 d = d0 + threadIdx.x;
    const u32 st = S.cnt[d], cn = S.cnt[d + 1] - st;
    const u32 pst = d ? S.cnt[d - 1] : 0u, pcn = st - pst;
    const bool f = d == 0 || st / T != pst / T || cn > T || pcn > T;
    const u32 bal = __ballot_sync(0xFFFFFFFFu, f);
    if ((threadIdx.x & 31) == 0) gflag[d >> 5] = bal;
    gstart[d] = st;
  }
  if (threadIdx.x == 0) gstart[kSubBins] = S.cnt[kSubBins];
  __syncthreads();
  for (u32 i = threadIdx.x; i < m; i += KB_BLOCK) {
    const u64 k = ak[base + i];
    const u64 d64 = (k - klo) >> sh;
    if (d64 >= (u64)kSubBins) continue;
    const u32 p = atomicAdd(&S.cnt[(u32)d64], 1u);
    if (p < m) {
      bk[base + p] = k;
      bv[base + p] = av[base + i];
    } else {
      flag_error(plan, ERR_INTERNAL);
    }
  }
  __syncthreads();
  // Pieces [d0, d1): from one flagged sub-bin to the next.
  u32 d0 = 0;
  while (d0 < (u32)kSubBins) {
    if (threadIdx.x == 0) {
      u32 d1 = d0 + 1;
      while (d1 < (u32)kSubBins) {
        const u32 w = gflag[d1 >> 5] >> (d1 & 31);
        if (w) { d1 += __ffs(w) - 1; break; }
        d1 = (d1 | 31u) + 1u;
      }
      S.misc[0] = d1 < (u32)kSubBins ? d1 : (u32)kSubBins;
    }
    __syncthreads();
    const u32 d1 = S.misc[0];
    const u32 ps = gstart[d0], pm = gstart[d1] - ps;
    __syncthreads();
#ifdef GBH_DEBUG_CHECKS
    if (ps + pm > m || d1 <= d0 || d1 > (u32)kSubBins) {
      if (threadIdx.x == 0) { DBG_REPORT(3, ps, pm, m, ((u64)d0 << 32) | d1); flag_error(plan, ERR_INTERNAL); }
      return;
    }
#endif
    if (pm > (u32)kGroupCap) {
      if (threadIdx.x == 0) flag_error(plan, ERR_FALLBACK);
      return;
    }
    if (pm > 0) {
      const u64 plo = klo + ((u64)d0 << sh);
      const bool binned = sort_into_smem<false>(S, bk, bv, base + ps, pm, plo, span_top(d1 - d0, sh), plan, DECIDE,
                                                Drop{nullptr, 0u, 0u, 0u}, rg);
      if (DECIDE) scan_piece(S, F, pm, base, plan->s, rg, plan, binned, plo);
      else write_out(S, bk, bv, base + ps, pm);
    }
    d0 = d1;
  }
}

// One block per group of consecutive bins, taken from a counter.  The
// survivors are in (ak, av), binned.  Without DECIDE the sorted result goes
// to (bk, bv).  With DECIDE (the hull pipeline) the second round runs on
// each sorted group at once, from the group's exclusive prefix in its
// record: only the kept points leave the block; the last block turns the
// groups' kept counts into offsets (then launch_group_compact).
template <bool DECIDE>
__global__ void __launch_bounds__(KB_BLOCK, KB_MIN_BLOCKS)
k3_bucket(const u64* __restrict__ ak, const u32* __restrict__ av, u64* bk, u32* bv, Plan* plan,
          const uint2* __restrict__ groups, u32* __restrict__ scratch, Fused F) {
  extern __shared__ __align__(16) unsigned char kb_smem[];
  BucketSmem& S = *reinterpret_cast<BucketSmem*>(kb_smem);
  __shared__ bool s_last;
  if (plan->error & (ERR_RANGE | ERR_FALLBACK)) return;
  const u32 ng = plan->ngroups;
  const u32 fshift = plan->fshift;
  const u32 s = plan->s;
  const RG rg = make_rg(plan);
  u32* my_scratch = scratch + (size_t)blockIdx.x * kScratchWords;
  // Thread 0 claims groups two ahead and fetches each descriptor one
  // group ahead (asynchronously, into shared memory), so that neither round
  // trip lies on the block's path.
  static_assert(offsetof(K4Chunk, inc_up) == offsetof(K4Chunk, inc_lo) + 8 && offsetof(K4Chunk, inc_lo) % 16 == 0,
                "prefix words fetched as one 16-byte copy");
  u32 g_next = 0;
  if (threadIdx.x == 0) {
    S.nerr = 0u;
    fetch_group<DECIDE>(S, F, groups, atomicAdd(&plan->ctr[CTR_BIN_GROUP], 1u), ng, plan);
    g_next = atomicAdd(&plan->ctr[CTR_BIN_GROUP], 1u);
  }
  for (;;) {
    if (threadIdx.x == 0) {
      cp_async_wait_all();
      const u32 g = (S.nerr & ERR_FALLBACK) ? ng : min(S.nid, ng);
      S.misc[1] = g;
      if (DECIDE && g < ng) start_group(S);
    }
    __syncthreads();
    const u32 g = S.misc[1];
    const uint2 a = S.nab[0], b = S.nab[1];   // (first position, first bin)
    __syncthreads();
    if (g >= ng) break;
    if (threadIdx.x == 0) {
      fetch_group<DECIDE>(S, F, groups, g_next, ng, plan);
      if (g_next < ng) g_next = atomicAdd(&plan->ctr[CTR_BIN_GROUP], 1u);
    }
    const u32 m = b.x - a.x;
#ifdef GBH_DEBUG_CHECKS
    if (b.x < a.x || b.x > s || b.y <= a.y || b.y > (u32)kBins) {
      if (threadIdx.x == 0) { DBG_REPORT(1, g, ng, ((u64)a.x << 32) | a.y, ((u64)b.x << 32) | b.y); flag_error(plan, ERR_INTERNAL); }
      break;
    }
#endif
    const u64 klo = (u64)a.y << fshift;
    const u32 span = fshift + ceil_log2(b.y - a.y);
    if (m <= (u32)kGroupCap) {
      if (m > 0) {
        const Drop dr{DECIDE ? F.bpre : nullptr, a.y, b.y - a.y, fshift};
        const bool binned = sort_into_smem<true>(S, ak, av, a.x, m, klo, span_top(b.y - a.y, fshift), plan, DECIDE,
                                                 dr, rg);
        const u32 mp = S.cnt[kSubBins];        // the pairs placed (all of them without the drop)
        if (threadIdx.x == 0) {      // the next group's pairs into L2 (its descriptor has arrived)
          cp_async_wait_all();
          if (S.nid < ng) {
            prefetch_span_l2(ak, S.nab[0].x, S.nab[1].x, sizeof(u64), 16u * kGroupCap);
            prefetch_span_l2(av, S.nab[0].x, S.nab[1].x, sizeof(u32), 8u * kGroupCap);
          }
        }
        if (DECIDE) scan_piece(S, F, mp, a.x, s, rg, plan, binned, klo);
        else write_out(S, bk, bv, a.x, m);
      }
    } else {
      big_bin<DECIDE>(S, ak, av, bk, bv, a.x, m, klo, span, my_scratch, plan, rg, F, g);
    }
    if (DECIDE && threadIdx.x == 0) {
      F.recs[g].cnt = make_uint2(S.kept[0], S.kept[1]);
      F.recs[g].base = a.x;
    }
  }
  if (!DECIDE) return;
  // The last block to finish turns the kept counts into offsets.
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(&plan->ctr[CTR_REGION2], 1u) == gridDim.x - 1;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  region_offsets(plan, F.recs, ng, s, &S.kwl[0][0], F.lo_xy, F.lo_idx, F.up_xy, F.up_idx);
}

// The second scatter of the bucket sort: spreads every coarse bin of
// (ak, av) over its kFinePerCoarse bins in (bk, bv).  Work comes in tiles
// of SP_TILE consecutive pairs of one coarse bin (tile ids in coarse-bin
// order, claimed from a counter one tile ahead).  A tile is ordered by bin
// in shared memory (counting), each of its bins reserves its run with one
// atomic on that bin's cursor (fcur, starting at the bin's first position;
// the reservation overlaps the placement), and the runs are written with
// consecutive threads on consecutive addresses.  With the tile ordered by
// bin, one warp per bin also folds the tile's points into the tile's
// direction aggregates of that bin: tagg[64 t + 2 d] (lower) and
// [64 t + 2 d + 1] (upper), 0 when the tile has no point of that bin and
// region; ctiles[c] = the first tile of coarse bin c (ctiles[kCoarse] = all
// tiles), written by block 0.
constexpr int SP_BLOCK = 512;
constexpr int SP_ITEMS = 8;
constexpr int SP_TILE = SP_BLOCK * SP_ITEMS;
constexpr int SP_WARPS = SP_BLOCK / 32;
static_assert(kFinePerCoarse == 32, "one lane per bin of a coarse bin");
static_assert(kCoarse <= SP_BLOCK, "one thread per coarse bin");
static_assert(SP_TILE <= 8192, "tile rank packed in 13 bits");
constexpr size_t SP_SMEM = (size_t)SP_TILE * (sizeof(u64) + sizeof(u32));

__global__ void __launch_bounds__(SP_BLOCK, 2)
k3_split(const u64* __restrict__ ak, const u32* __restrict__ av, u64* __restrict__ bk, u32* __restrict__ bv,
         Plan* plan, const u32* __restrict__ bstart, u32* __restrict__ fcur, u64* __restrict__ tagg,
         u32* __restrict__ ctiles) {
  extern __shared__ __align__(16) unsigned char sp_smem[];   // SP_TILE keys, then SP_TILE indices
  u64* s_key = reinterpret_cast<u64*>(sp_smem);
  u32* s_idx = reinterpret_cast<u32*>(sp_smem + SP_TILE * sizeof(u64));
  __shared__ u32 s_tiles[kCoarse + 1];
  __shared__ u32 s_cnt[kFinePerCoarse], s_lst[kFinePerCoarse + 1], s_gb[kFinePerCoarse];
  __shared__ u32 s_w[SP_WARPS];
  __shared__ u32 s_t, s_c;
  if (plan->error & (ERR_RANGE | ERR_FALLBACK)) return;
  const u32 s = plan->s, fshift = plan->fshift;
  const RG rg = make_rg(plan);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const u64 pol_in = policy_evict_first();    // the coarse bins are dead once split
  u32 t_next = 0;
  if (threadIdx.x == 0) t_next = atomicAdd(&plan->ctr[CTR_SPLIT], 1u);
  // Tiles per coarse bin and their exclusive prefix.
  u32 nt = 0;
  if (threadIdx.x < kCoarse) {
    const u32 c = threadIdx.x;
    const u32 cs = bstart[c * kFinePerCoarse];
    const u32 ce = c + 1 < (u32)kCoarse ? bstart[(c + 1) * kFinePerCoarse] : s;
    nt = (ce - cs + SP_TILE - 1) / SP_TILE;
  }
  u32 inc = nt;
  #pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const u32 t = __shfl_up_sync(0xFFFFFFFFu, inc, o);
    if (lane >= o) inc += t;
  }
  if (lane == 31) s_w[wid] = inc;
  __syncthreads();
  u32 off = 0, tot = 0;
  for (int w = 0; w < SP_WARPS; ++w) {
    if (w < wid) off += s_w[w];
    tot += s_w[w];
  }
  if (threadIdx.x < kCoarse) {
    s_tiles[threadIdx.x] = off + inc - nt;
    if (blockIdx.x == 0) ctiles[threadIdx.x] = off + inc - nt;
  }
  if (threadIdx.x == 0) {
    s_tiles[kCoarse] = tot;
    if (blockIdx.x == 0) ctiles[kCoarse] = tot;
  }
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) {
      const u32 t = t_next;
      s_t = t;
      if (t < tot) {
        t_next = atomicAdd(&plan->ctr[CTR_SPLIT], 1u);
        u32 lo = 0, hi = kCoarse - 1;       // largest c with s_tiles[c] <= t
        while (lo < hi) {
          const u32 mid = (lo + hi + 1) >> 1;
          if (s_tiles[mid] <= t) lo = mid; else hi = mid - 1;
        }
        s_c = lo;
      }
    }
    if (threadIdx.x < kFinePerCoarse) s_cnt[threadIdx.x] = 0u;
    __syncthreads();
    const u32 t = s_t;
    if (t >= tot) break;
    const u32 c = s_c;
    const u32 cs = bstart[c * kFinePerCoarse];
    const u32 ce = c + 1 < (u32)kCoarse ? bstart[(c + 1) * kFinePerCoarse] : s;
    const u32 start = cs + (t - s_tiles[c]) * (u32)SP_TILE;
    const u32 n = start < ce ? min((u32)SP_TILE, ce - start) : 0u;
    u64 key[SP_ITEMS];
    u32 idx[SP_ITEMS], pk[SP_ITEMS];
    // The tile's pairs are loaded together, then counted.
    #pragma unroll
    for (int it = 0; it < SP_ITEMS; ++it) {
      const u32 i = it * SP_BLOCK + threadIdx.x;
      key[it] = 0ull;
      idx[it] = 0u;
      if (i < n) {
        key[it] = ld_hint_u64(ak + start + i, pol_in);
        idx[it] = ld_hint_u32(av + start + i, pol_in);
      }
    }
    #pragma unroll
    for (int it = 0; it < SP_ITEMS; ++it) {
      const u32 i = it * SP_BLOCK + threadIdx.x;
      pk[it] = 0xFFFFFFFFu;
      if (i < n) {
        const u32 f = (u32)(key[it] >> fshift);
        if ((f >> (kBinBits - kCoarseBits)) == c) {
          const u32 d = f & (kFinePerCoarse - 1);
          pk[it] = (d << 13) | atomicAdd(&s_cnt[d], 1u);
        } else {
          flag_error(plan, ERR_INTERNAL);
        }
      }
    }
    __syncthreads();
    u32 gb = 0;
    if (wid == 0) {
      const u32 cn = s_cnt[lane];
      u32 x = cn;
      #pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const u32 y = __shfl_up_sync(0xFFFFFFFFu, x, o);
        if (lane >= o) x += y;
      }
      s_lst[lane] = x - cn;
      if (lane == 31) s_lst[kFinePerCoarse] = x;
      gb = cn ? atomicAdd(&fcur[c * kFinePerCoarse + lane], cn) : 0u;   // used after the placement
    }
    __syncthreads();
    #pragma unroll
    for (int it = 0; it < SP_ITEMS; ++it) {
      if (pk[it] != 0xFFFFFFFFu) {
        const u32 p = s_lst[pk[it] >> 13] + (pk[it] & 8191u);
        s_key[p] = key[it];
        s_idx[p] = idx[it];
      }
    }
    if (wid == 0) s_gb[lane] = gb;
    __syncthreads();
    const u32 placed = s_lst[kFinePerCoarse];
    for (u32 j = threadIdx.x; j < placed; j += SP_BLOCK) {
      const u64 k = s_key[j];
      const u32 d = (u32)(k >> fshift) & (kFinePerCoarse - 1);
      const u32 pos = s_gb[d] + (j - s_lst[d]);
      if (pos < s) {
        bk[pos] = k;
        bv[pos] = s_idx[j];
      } else {
        flag_error(plan, ERR_INTERNAL);
      }
    }
    // Half a warp per bin: the tile's aggregates of the bin (plain stores;
    // a word without its valid bit holds nothing).
    static_assert(2 * SP_WARPS == kFinePerCoarse, "two bins per warp");
    {
      const u32 d = 2 * wid + (lane >> 4), h = lane & 15;
      const u32 a = s_lst[d], b = s_lst[d + 1];
      Dir2 v = rg.ident;
      for (u32 j = a + h; j < b; j += 16) add_dir(v, rg, s_key[j]);
      #pragma unroll
      for (int o = 8; o > 0; o >>= 1) combine(v, shfl_xor_dir(v, o));
      u64* w = tagg + (size_t)t * (2 * kFinePerCoarse) + 2 * d;
      if (h == 0) w[0] = (v.lx != rg.ident.lx || v.ly != rg.ident.ly) ? pack_dir(v.lx, v.ly) : 0ull;
      if (h == 1) w[1] = (v.ux != rg.ident.ux || v.uy != rg.ident.uy) ? pack_dir(v.ux, v.uy) : 0ull;
    }
  }
}

// Exclusive prefixes of the bins' direction aggregates.  Block k owns
// bins [k BP_BLOCK, (k + 1) BP_BLOCK): thread b folds bin b's tile
// aggregates (tagg, ctiles from k3_split), the block scans its bins and
// writes each bin's prefix within the block to bagg and the block's total
// after the kBins bins.  The last block scans the block totals and combines
// each bin's prefix within its block with the totals of the blocks before
// it: bin b's words of bpre receive the extreme of the directions of every
// point in bins 0 .. b - 1 together with d(P_0) (the identity), lower and
// upper region, and record g's prefix words the prefix of its first bin.
constexpr int BP_BLOCK = 512;
constexpr int BP_GRID = kBins / BP_BLOCK;
constexpr int BP_WARPS = BP_BLOCK / 32;
constexpr int BP_PER = kBins / BP_BLOCK;   // bins per thread in the last block
static_assert(BP_GRID * BP_BLOCK == kBins && BP_GRID <= 32 && BP_GRID <= kBinPrefixBlocks, "one lane per block total");
static_assert(BP_PER % 8 == 0, "whole batches of eight");

__global__ void __launch_bounds__(BP_BLOCK)
k_bin_prefix(Plan* plan, K4Chunk* __restrict__ recs, const uint2* __restrict__ groups,
             const u64* __restrict__ tagg, const u32* __restrict__ ctiles, u64* __restrict__ bagg,
             u64* __restrict__ bpre) {
  __shared__ bool s_last;
  __shared__ Dir2 s_w[BP_WARPS];
  __shared__ Dir2 s_bx[BP_GRID];            // last block: exclusive prefixes of the block totals
  if (plan->error & (ERR_RANGE | ERR_FALLBACK)) return;
  const RG rg = make_rg(plan);
  ulonglong2* a2 = reinterpret_cast<ulonglong2*>(bagg);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  {
    const u32 b = blockIdx.x * BP_BLOCK + threadIdx.x;
    const u32 c = b / kFinePerCoarse, d = b % kFinePerCoarse;
    const u32 t0 = ctiles[c], t1 = ctiles[c + 1];
    Dir2 v = rg.ident;
    for (u32 tb = t0; tb < t1; tb += 8) {       // eight tiles' words loaded together
      u64 wv[16];
      #pragma unroll
      for (int k = 0; k < 8; ++k) {
        const u64* w = tagg + (size_t)(tb + k) * (2 * kFinePerCoarse) + 2 * d;
        wv[2 * k] = tb + k < t1 ? w[0] : 0ull;
        wv[2 * k + 1] = tb + k < t1 ? w[1] : 0ull;
      }
      #pragma unroll
      for (int k = 0; k < 8; ++k) combine(v, unpack_pair(wv[2 * k], wv[2 * k + 1], rg));
    }
    const Dir2 inc = warp_scan_dir(v);
    const Dir2 lex = shfl_up_dir(inc, 1);
    if (lane == 31) s_w[wid] = inc;
    __syncthreads();
    Dir2 e = rg.ident;
    for (int w = 0; w < wid; ++w) combine(e, s_w[w]);
    if (threadIdx.x == BP_BLOCK - 1) {           // the block's total
      Dir2 tot = e;
      combine(tot, inc);
      a2[kBins + blockIdx.x] = make_ulonglong2(pack_dir(tot.lx, tot.ly), pack_dir(tot.ux, tot.uy));
    }
    if (lane > 0) combine(e, lex);
    a2[b] = make_ulonglong2(pack_dir(e.lx, e.ly), pack_dir(e.ux, e.uy));
  }
  if (!last_block(plan, CTR_GROUP_AGG, &s_last)) return;
  // (L2 loads: the prefixes come from other blocks)
  if (wid == 0) {
    Dir2 t = rg.ident;
    if (lane < BP_GRID) {
      const ulonglong2 w = __ldcg(&a2[kBins + lane]);
      t = unpack_pair(w.x, w.y, rg);
    }
    const Dir2 inc = warp_scan_dir(t);
    Dir2 ex = shfl_up_dir(inc, 1);
    if (lane == 0) ex = rg.ident;
    if (lane < BP_GRID) s_bx[lane] = ex;
  }
  __syncthreads();
  const u32 ng = plan->ngroups;
  for (u32 g0 = threadIdx.x; g0 < ng; g0 += 8 * BP_BLOCK) {   // eight groups per thread at a time
    u32 fb[8];
    #pragma unroll
    for (int k = 0; k < 8; ++k) {
      const u32 g = g0 + k * BP_BLOCK;
      fb[k] = g < ng ? groups[g].y : 0u;
    }
    ulonglong2 wv[8];
    #pragma unroll
    for (int k = 0; k < 8; ++k) wv[k] = __ldcg(&a2[fb[k]]);
    #pragma unroll
    for (int k = 0; k < 8; ++k) {
      const u32 g = g0 + k * BP_BLOCK;
      if (g < ng) {
        Dir2 e = s_bx[fb[k] / BP_BLOCK];
        combine(e, unpack_pair(wv[k].x, wv[k].y, rg));
        recs[g].inc_lo = pack_dir(e.lx, e.ly);
        recs[g].inc_up = pack_dir(e.ux, e.uy);
      }
    }
  }
  ulonglong2* p2 = reinterpret_cast<ulonglong2*>(bpre);
  for (int k0 = 0; k0 < BP_PER; k0 += 8) {     // bin k BP_BLOCK + t: block k's prefix, then its own
    ulonglong2 wv[8];
    #pragma unroll
    for (int k = 0; k < 8; ++k) wv[k] = __ldcg(&a2[(k0 + k) * BP_BLOCK + threadIdx.x]);
    #pragma unroll
    for (int k = 0; k < 8; ++k) {
      Dir2 e = s_bx[k0 + k];
      combine(e, unpack_pair(wv[k].x, wv[k].y, rg));
      p2[(k0 + k) * BP_BLOCK + threadIdx.x] = make_ulonglong2(pack_dir(e.lx, e.ly), pack_dir(e.ux, e.uy));
    }
  }
}

// Bin starts and groups of the array path (the stage entry point; the
// pipeline's come from the fused filter's last block).  k_binscan takes one
// histogram row per histogram block: row r, bin b becomes the number of
// bin-b pairs of rows before r, bstart[b] first receives the bin totals, and
// its last block writes the bins' first positions and the groups (first
// position, first bin), with a closing record (s, kBins) after the last
// group (bins_to_groups, bins.cuh).
constexpr int BS_BINS = 32;                 // bins per block (one per lane)
constexpr int BS_RMAX = 10;                 // rows a warp loads at once

__global__ void __launch_bounds__(BS_BLOCK)
k_binscan(u32* __restrict__ rows, u32 nrows, Plan* plan, u32* __restrict__ bstart,
          uint2* __restrict__ groups, u32* __restrict__ fcur) {
  __shared__ u32 s_part[BS_WARPS][BS_BINS];
  __shared__ bool s_last;
  if (plan->error & ERR_RANGE) return;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const u32 bin = blockIdx.x * BS_BINS + lane;
  const u32 per = (nrows + BS_WARPS - 1) / BS_WARPS;
  const u32 r0 = min(nrows, wid * per), r1 = min(nrows, r0 + per);
  u32 sum = 0;
  for (u32 rb = r0; rb < r1; rb += BS_RMAX) {       // the rows of a batch are loaded together
    u32 v[BS_RMAX];
    #pragma unroll
    for (int q = 0; q < BS_RMAX; ++q) v[q] = rb + q < r1 ? rows[(size_t)(rb + q) * kBins + bin] : 0u;
    #pragma unroll
    for (int q = 0; q < BS_RMAX; ++q) sum += v[q];
  }
  s_part[wid][lane] = sum;
  __syncthreads();
  u32 run = 0, tot = 0;
  for (int w = 0; w < BS_WARPS; ++w) {
    if (w < wid) run += s_part[w][lane];
    tot += s_part[w][lane];
  }
  for (u32 rb = r0; rb < r1; rb += BS_RMAX) {
    u32 v[BS_RMAX];
    #pragma unroll
    for (int q = 0; q < BS_RMAX; ++q) v[q] = rb + q < r1 ? rows[(size_t)(rb + q) * kBins + bin] : 0u;
    #pragma unroll
    for (int q = 0; q < BS_RMAX; ++q) {
      if (rb + q < r1) rows[(size_t)(rb + q) * kBins + bin] = run;
      run += v[q];
    }
  }
  if (wid == 0) bstart[bin] = tot;

  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(&plan->ctr[CTR_BIN_SCAN], 1u) == gridDim.x - 1;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  __shared__ BinScanSmem B;
  bins_to_groups<true>(bstart, plan, bstart, groups, fcur, B);
}

// ---- the same sort over an arbitrary key array (the stage entry point):
// key bits from an OR of all keys, then per-block bin rows over chunks of
// KA_CHUNK keys (chunk c in block c mod grid), the bin scan, and a scatter
// over the same chunks.
constexpr int KA_BLOCK = 256;
constexpr int KA_CHUNK = 4096;

__global__ void __launch_bounds__(KA_BLOCK)
k3_array_keyor(const u64* __restrict__ keys, Plan* plan, unsigned long long* key_or) {
  const u32 s = plan->s;
  u64 v = 0;
  for (u32 i = blockIdx.x * KA_BLOCK + threadIdx.x; i < s; i += gridDim.x * KA_BLOCK) v |= keys[i];
  #pragma unroll
  for (int o = 16; o > 0; o >>= 1) v |= __shfl_xor_sync(0xFFFFFFFFu, v, o);
  if ((threadIdx.x & 31) == 0 && v) atomicOr(key_or, (unsigned long long)v);
}

__global__ void __launch_bounds__(KA_BLOCK)
k3_array_hist(const u64* __restrict__ keys, Plan* plan, const unsigned long long* key_or,
              u32* __restrict__ rows) {
  extern __shared__ u32 h[];
  const u32 s = plan->s;
  const u64 o = *key_or;
  const u32 kbits = o ? 64u - (u32)__clzll((long long)o) : 0u;
  const u32 fshift = kbits > (u32)kBinBits ? kbits - (u32)kBinBits : 0u;
  if (blockIdx.x == 0 && threadIdx.x == 0) plan->fshift = fshift;
  for (u32 q = threadIdx.x; q < (u32)kBins; q += KA_BLOCK) h[q] = 0u;
  __syncthreads();
  for (u32 c = blockIdx.x; (size_t)c * KA_CHUNK < s; c += gridDim.x)
    for (u32 i = c * KA_CHUNK + threadIdx.x; i < min(s, (c + 1) * (u32)KA_CHUNK); i += KA_BLOCK)
      atomicAdd(&h[(u32)(keys[i] >> fshift)], 1u);
  __syncthreads();
  for (u32 q = threadIdx.x; q < (u32)kBins; q += KA_BLOCK) rows[(size_t)blockIdx.x * kBins + q] = h[q];
}

__global__ void __launch_bounds__(KA_BLOCK)
k3_array_scatter(const u64* __restrict__ keys, const u32* __restrict__ vals, Plan* plan,
                 const u32* __restrict__ rows, const u32* __restrict__ bstart, u64* __restrict__ ok,
                 u32* __restrict__ ov) {
  extern __shared__ u32 cur[];
  const u32 s = plan->s;
  const u32 fshift = plan->fshift;
  for (u32 q = threadIdx.x; q < (u32)kBins; q += KA_BLOCK)
    cur[q] = bstart[q] + rows[(size_t)blockIdx.x * kBins + q];
  __syncthreads();
  for (u32 c = blockIdx.x; (size_t)c * KA_CHUNK < s; c += gridDim.x)
    for (u32 i = c * KA_CHUNK + threadIdx.x; i < min(s, (c + 1) * (u32)KA_CHUNK); i += KA_BLOCK) {
      const u64 k = keys[i];
      const u32 p = atomicAdd(&cur[(u32)(k >> fshift)], 1u);
      if (p < s) { ok[p] = k; ov[p] = vals[i]; }
      else flag_error(plan, ERR_INTERNAL);
    }
}

#ifdef GBH_DEBUG_CHECKS
// Region lists must be strictly increasing in (x, y) from P_0 to P_l.
__global__ void k_check_regions(const Plan* plan, const int2* lo_xy, const int2* up_xy) {
  for (int c = 0; c < 2; ++c) {
    const int2* L = c ? up_xy : lo_xy;
    const u32 r = c ? plan->r_up : plan->r_lo;
    if (r > plan->s) { if (threadIdx.x == 0 && blockIdx.x == 0) DBG_REPORT(10 + c, r, plan->s, 0, 0); return; }
    for (u32 i = blockIdx.x * blockDim.x + threadIdx.x; i + 1 < r + 2; i += gridDim.x * blockDim.x) {
      const int2 p = L[i], q = L[i + 1];
      if (!(p.x < q.x || (p.x == q.x && p.y < q.y))) DBG_REPORT(20 + c, i, r, ((u64)(u32)p.x << 32) | (u32)p.y, ((u64)(u32)q.x << 32) | (u32)q.y);
    }
  }
}
#endif

}  // namespace

#ifdef GBH_DEBUG_CHECKS
cudaError_t launch_check_regions(const Plan* plan, const int2* lo_xy, const int2* up_xy, cudaStream_t st) {
  k_check_regions<<<64, 256, 0, st>>>(plan, lo_xy, up_xy);
  return cudaGetLastError();
}
#endif

size_t bucket_smem() { return sizeof(BucketSmem); }
size_t bucket_scratch_words(int blocks) { return (size_t)blocks * kScratchWords; }

cudaError_t bucket_configure() {
  cudaError_t e = cudaFuncSetAttribute(k3_bucket<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)sizeof(BucketSmem));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k3_bucket<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(BucketSmem));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k3_split, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SP_SMEM);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k3_array_hist, cudaFuncAttributeMaxDynamicSharedMemorySize, kBins * 4);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k3_array_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize, kBins * 4);
  return e;
}

cudaError_t bucket_occupancy(int* blocks) {
  int a = 0, b = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k3_bucket<false>, KB_BLOCK, sizeof(BucketSmem));
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k3_bucket<true>, KB_BLOCK, sizeof(BucketSmem));
  *blocks = a < b ? a : b;
  return e;
}



cudaError_t launch_bucket_sort(const u64* ak, const u32* av, u64* bk, u32* bv, Plan* plan,
                               const uint2* groups, u32* scratch, int grid, cudaStream_t st) {
  Fused F{};
  k3_bucket<false><<<grid, KB_BLOCK, sizeof(BucketSmem), st>>>(ak, av, bk, bv, plan, groups, scratch, F);
  return cudaGetLastError();
}

cudaError_t launch_split(const u64* ak, const u32* av, u64* bk, u32* bv, Plan* plan, const u32* bstart, u32* fcur,
                         u64* tagg, u32* ctiles, int grid, cudaStream_t st) {
  k3_split<<<grid, SP_BLOCK, SP_SMEM, st>>>(ak, av, bk, bv, plan, bstart, fcur, tagg, ctiles);
  return cudaGetLastError();
}

int split_tile() { return SP_TILE; }

cudaError_t split_occupancy(int* blocks) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, k3_split, SP_BLOCK, SP_SMEM);
}

cudaError_t launch_bin_prefix(Plan* plan, const uint2* groups, void* recs, const u64* tagg, const u32* ctiles,
                              u64* bagg, u64* bpre, cudaStream_t st) {
  k_bin_prefix<<<kBins / BP_BLOCK, BP_BLOCK, 0, st>>>(plan, reinterpret_cast<K4Chunk*>(recs), groups, tagg, ctiles,
                                                      bagg, bpre);
  return cudaGetLastError();
}

cudaError_t launch_bucket_decide(const u64* ak, const u32* av, u64* bk, u32* bv, Plan* plan, const uint2* groups,
                                 u32* scratch, void* recs, const u64* bpre, int2* t_lo_xy, int* t_lo_idx,
                                 int2* t_up_xy, int* t_up_idx, int2* lo_xy, int* lo_idx, int2* up_xy, int* up_idx,
                                 int grid, cudaStream_t st) {
  Fused F{reinterpret_cast<K4Chunk*>(recs), t_lo_xy, t_lo_idx, t_up_xy, t_up_idx, lo_xy, lo_idx, up_xy, up_idx, bpre};
  k3_bucket<true><<<grid, KB_BLOCK, sizeof(BucketSmem), st>>>(ak, av, bk, bv, plan, groups, scratch, F);
  return cudaGetLastError();
}

int array_hist_grid(u32 m, int num_sms) {
  const u32 chunks = (m + KA_CHUNK - 1) / KA_CHUNK;
  const u32 g = (u32)num_sms * 2u;
  return (int)(chunks < 1 ? 1 : (chunks < g ? chunks : g));
}

cudaError_t launch_array_bins(const u64* keys, const u32* vals, u32 m, Plan* plan,
                              unsigned long long* key_or, u32* rows, u32* bstart, uint2* groups,
                              u64* ok, u32* ov, int grid, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(key_or, 0, sizeof(unsigned long long), st);
  if (e != cudaSuccess) return e;
  k3_array_keyor<<<grid, KA_BLOCK, 0, st>>>(keys, plan, key_or);
  k3_array_hist<<<grid, KA_BLOCK, kBins * 4, st>>>(keys, plan, key_or, rows);
  k_binscan<<<kBins / BS_BINS, BS_BLOCK, 0, st>>>(rows, (u32)grid, plan, bstart, groups, nullptr);
  k3_array_scatter<<<grid, KA_BLOCK, kBins * 4, st>>>(keys, vals, plan, rows, bstart, ok, ov);
  (void)m;
  return cudaGetLastError();
}

}  // namespace gbh
