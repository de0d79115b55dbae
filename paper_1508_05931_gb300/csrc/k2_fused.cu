// The pipeline's front after K1, in one pass over the points: the
// first-round filter (Section 2.1 step 2, Section 3.1) and the test of the
// second round (Section 2.2, Figure 2) against a witness from a sample,
// fused with the compaction of what is left.
//
// Figure 2 walks each region in sort order and keeps a point exactly when
// its direction from P_l is strictly beyond the running extreme P_temp of
// the first-round survivors before it (reading 14: an exclusive prefix
// extreme).  Any first-round survivor w that precedes p in sort order and
// lies in p's region is part of that running extreme, so a point whose
// direction is not strictly beyond w's is discarded by Figure 2 wherever it
// stands, and leaves the running extreme of every later point unchanged.
// Removing such points before the sort keeps the second round's lists
// exactly as Figure 2 computes them; the sort's own early drop (k3_bucket.cu)
// rests on the same argument.  A point is passed on only when it survives
// both tests; the order of the two tests is free.
//
//   k_witness  reads the sample of every kSampleStride-th point (copied out
//              by K1), or on the single-read front the raw survivors of
//              the sample polygon (the points nearest the hull; every st-th
//              of them when they outnumber that sample); a point
//              that survives the filter polygon and lies off the line
//              P_0 P_l is a witness for every later witness bin (the top
//              kWitnessBits of the key) of its region.
//              Per witness bin and region the sample's most advanced
//              direction is kept by one 64-bit atomic maximum of (a monotone
//              float pseudo-angle, sample index + 1).  The pseudo-angle only
//              chooses among valid witnesses, so its rounding can cost a
//              little discarding, never exactness.
//   k2_fused   (one block per SM) first turns those maxima into every
//              witness bin's exclusive prefix, a table of witness directions
//              in shared memory (the direction of P_0 - P_l where no sample
//              point precedes).  Every point then meets the witness test of
//              its bin and region (exact int64, one shared-memory lookup);
//              the few that pass are staged per warp, and when a warp flushes
//              its slice they meet the filter polygon (exact int64, points
//              decoded from their keys) and the rest go to the output with
//              one atomic reservation per flush (the order of the output is
//              free: the bucket sort orders (key, index) pairs itself), their
//              bins' totals to btot.  The polygon test, the costlier of the
//              two, thus runs on about one point in fifty.  With COUNT the
//              polygon is also tested on every point, to count the
//              first-round survivors for the statistics.  The last block to
//              finish turns the bins' totals into bin starts and groups
//              (bins_to_groups, in the table's shared memory, free by then).
//   k2_place   after the bin scan, moves the output into coarse-bin order
//              (one reservation per coarse bin and chunk), the input of
//              k3_split.
// Points on the line P_0 P_l pass the witness test: the region split drops
// them.
#include <cstddef>

#include "bins.cuh"
#include "filter.cuh"
#include "hull_internal.cuh"
#include "kernels.h"
#include "regions.cuh"

namespace gbh {

namespace {

// Pseudo-angle of direction d = p - P_l in its region, increasing towards
// the direction Figure 2 keeps: with c = cross(P_0 - P_l, d) (> 0 lower,
// < 0 upper) and e = dot(P_0 - P_l, d), q = 1 - e / (|e| + |c|) runs from 0
// (along P_0 - P_l) through 1 (perpendicular) to 2 (opposite), monotone in
// the angle between P_0 - P_l and d on either side.  Quantised to 32 bits.
__device__ __forceinline__ u32 pseudo_angle(long long c, long long e) {
  const float fc = fabsf((float)c), fe = (float)e;
  const float q = 1.0f - fe / (fabsf(fe) + fc);
  return (u32)fminf(fmaxf(q, 0.0f) * 2147483648.0f, 4294967040.0f);
}

__device__ __forceinline__ u32 witness_shift(const Plan* plan) {
  return plan->kbits > (u32)kWitnessBits ? plan->kbits - (u32)kWitnessBits : 0u;
}

constexpr int SW_BLOCK = 256;
constexpr int SW_ITEMS = 4;                   // sampled points per thread and round, loaded together

__global__ void __launch_bounds__(SW_BLOCK)
k_witness(const int2* __restrict__ sample, Plan* plan, u64* __restrict__ wkey, const u32* __restrict__ ncount) {
  if (plan->error & ERR_RANGE) return;
  const u32 n = plan->n;
  // The candidates: sample[0, S) with a stride; with ncount, at most as
  // many as the every-32nd-point sample would hold (every st-th raw
  // survivor when there are more: any subset of the first-round survivors
  // gives valid witnesses).
  const u32 cap = (n + kSampleStride - 1) / kSampleStride;
  const u32 R = ncount ? *ncount : cap;
  const u32 st = R > cap ? (R + cap - 1) / cap : 1u;
  const u32 S = (R + st - 1) / st;
  const int K = plan->ncorner;
  Edges E;
  load_edges(plan, K, E);
  const int bx = plan->ext_x[1], by = plan->ext_y[1];
  const int ux = plan->ext_x[0] - bx, uy = plan->ext_y[0] - by;   // P_0 - P_l
  const int x0 = plan->key_x0, y0 = plan->key_y0;
  const u32 ybits = plan->ybits, wshift = witness_shift(plan);
  const u32 T = gridDim.x * SW_BLOCK;
  for (u32 i0 = blockIdx.x * SW_BLOCK + threadIdx.x; i0 < S; i0 += SW_ITEMS * T) {
    int2 p[SW_ITEMS];
    #pragma unroll
    for (int q = 0; q < SW_ITEMS; ++q) p[q] = i0 + q * T < S ? sample[(i0 + q * T) * st] : make_int2(0, 0);
    #pragma unroll
    for (int q = 0; q < SW_ITEMS; ++q) {
      const u32 i = (i0 + q * T) * st;    // the candidate's position in sample[]
      if (i0 + q * T >= S || strictly_inside_rt(E, K, p[q].x, p[q].y)) continue;   // not a first-round survivor
      const int dx = p[q].x - bx, dy = p[q].y - by;
      const long long c = cross2(ux, uy, dx, dy);
      if (c == 0) continue;                                             // on the line P_0 P_l: no region
      const long long e = (long long)ux * dx + (long long)uy * dy;
      const u64 key = ((u64)(u32)(p[q].x - x0) << ybits) | (u64)(u32)(p[q].y - y0);
      const u32 wb = (u32)(key >> wshift);
      atomicMax(&wkey[(c > 0 ? 0u : (u32)kWitnessBins) + wb], ((u64)pseudo_angle(c, e) << 32) | (u64)(i + 1u));
    }
  }
}

// ---- k2_fused
// One block per SM with its copy of the witness table; every thread streams
// the points with 128-bit loads, KF_V at a time, the next round's loads
// issued before the current round is tested (the registers this takes are
// why the block has the SM to itself: 116 a thread).  A warp
// stages the points that pass the witness test in its own slice of the
// staging area (no block-wide barrier in the stream) and flushes the slice
// by itself when the next batch would not fit, and at the end.
constexpr int KF_BLOCK = 512;
constexpr int KF_WARPS = KF_BLOCK / 32;
#ifndef KF_V_CFG
#define KF_V_CFG 4
#endif
#ifndef KF_PF_CFG
#define KF_PF_CFG 1
#endif
#ifndef KF_MINB_CFG
#define KF_MINB_CFG 1
#endif
constexpr int KF_V = KF_V_CFG;                         // int4 (two points) per thread per round
constexpr bool KF_PF = KF_PF_CFG != 0;                 // load the next full round before computing this one
#ifndef KF_CONTIG_CFG
#define KF_CONTIG_CFG 1
#endif
constexpr bool KF_CONTIG = KF_CONTIG_CFG != 0;      // every warp reads one contiguous run per round
// (Measured: 62.7 / 60.6 us per launch on the 20M square / disk against
// 65.1 / 63.5 with slot r of all threads contiguous instead.)
// (Measured on the 20M square and disk: 65 / 64 us a launch against 70 / 69
// for two blocks per SM at 64 registers without the early loads.)
constexpr int KF_PTS = 2 * KF_V;                       // points per thread per round
constexpr int KF_SLICE = 256;                          // staged points per warp: at least a whole round of survivors
static_assert(KF_SLICE >= 32 * KF_PTS, "a round's survivors fit a slice");
constexpr int KF_WPER = (kWitnessBins + KF_BLOCK - 1) / KF_BLOCK;   // witness bins per thread in the prologue
struct KFEdge {
  int ex, ney;
  long long nc;               // orient(c_j, c_j+1, p) = ex y + ney x + nc
};
struct KFSmem {
  int2 wt[2 * kWitnessBins];                           // witness direction of (bin, region)
  u64 key[KF_WARPS][KF_SLICE];
  u32 idx[KF_WARPS][KF_SLICE];
  KFEdge edge[kMaxCorners];                            // the filter polygon
  int ncorner;
};
constexpr size_t KF_SMEM = sizeof(KFSmem);

struct Front {
  int bx, by, ux, uy;         // P_l and P_0 - P_l
  int x0, y0;                 // key origin
  u32 ybits, fshift;          // key layout, sort bins
  u32 s1, s2, ysh;            // witness bin = ((x - x0) << s2 >> s1) | ((y - y0) >> ysh)
  u64 ymask;
};

__device__ __forceinline__ Front make_front(const Plan* plan) {
  Front F;
  F.bx = plan->ext_x[1]; F.by = plan->ext_y[1];
  F.ux = plan->ext_x[0] - F.bx; F.uy = plan->ext_y[0] - F.by;
  F.x0 = plan->key_x0; F.y0 = plan->key_y0;
  F.ybits = plan->ybits; F.fshift = plan->fshift;
  F.ymask = F.ybits ? ((~0ull) >> (64 - F.ybits)) : 0ull;
  const u32 w = witness_shift(plan);
  // key >> w in 32-bit pieces: the x part (x - x0) << ybits >> w, the y part
  // (y - y0) >> w (zero once w >= ybits, as y - y0 < 2^ybits).
  F.s1 = w >= F.ybits ? w - F.ybits : 0u;
  F.s2 = w >= F.ybits ? 0u : F.ybits - w;
  F.ysh = w < 31u ? w : 31u;
  return F;
}

// Witness test of one point inside the bounding box; true: it passes.
// XONLY: the witness bin is (x - x0) >> s1 (the key's x part alone covers
// the witness bits).  The point passes when it lies on P_0 P_l (c = 0), or
// when c and t = cross(w, d) are nonzero with the same sign (lower region
// c > 0: strictly counter-clockwise of the witness; upper c < 0: strictly
// clockwise).
template <bool XONLY>
__device__ __forceinline__ bool witness_pass(const Front& F, const int2* wt, int x, int y) {
  const int dx = x - F.bx, dy = y - F.by;
  const long long c = cross2(F.ux, F.uy, dx, dy);
  const u32 wb = XONLY ? (u32)(x - F.x0) >> F.s1
                       : (((u32)(x - F.x0) << F.s2) >> F.s1) | ((u32)(y - F.y0) >> F.ysh);
  const u32 chi = (u32)((unsigned long long)c >> 32);
  const int2 w = wt[(wb << 1) | (chi >> 31)];
  const long long t = cross2(w.x, w.y, dx, dy);
  const u32 thi = (u32)((unsigned long long)t >> 32);
  return c == 0 || ((int)(chi ^ thi) >= 0 && t != 0);
}

// The witness table of the block (every thread of the block calls it):
// thread t owns witness bins [t KF_WPER, (t + 1) KF_WPER) of both regions.
__device__ void build_witness_table(const u64* __restrict__ wkey, const int2* __restrict__ sample, const Front& F,
                                    KFSmem& S, u64* s_wm) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int r = 0; r < 2; ++r) {
    u64 v[KF_WPER];
    const u32 b0 = threadIdx.x * KF_WPER;        // bins past kWitnessBins are empty
    #pragma unroll
    for (int q = 0; q < KF_WPER; ++q) v[q] = b0 + q < (u32)kWitnessBins ? __ldcg(&wkey[(size_t)r * kWitnessBins + b0 + q]) : 0ull;
    u64 tot = 0;
    #pragma unroll
    for (int q = 0; q < KF_WPER; ++q) tot = v[q] > tot ? v[q] : tot;
    u64 inc = tot;
    #pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const u64 t = __shfl_up_sync(0xFFFFFFFFu, inc, o);
      if (lane >= o && t > inc) inc = t;
    }
    u64 ex = __shfl_up_sync(0xFFFFFFFFu, inc, 1);
    if (lane == 0) ex = 0;
    if (lane == 31) s_wm[wid] = inc;
    __syncthreads();
    for (int w = 0; w < wid; ++w) ex = s_wm[w] > ex ? s_wm[w] : ex;
    u32 widx[KF_WPER];
    #pragma unroll
    for (int q = 0; q < KF_WPER; ++q) {
      widx[q] = (u32)ex;                     // sample index + 1 of the witness, 0: none
      ex = v[q] > ex ? v[q] : ex;
    }
    // Consecutive bins mostly share their witness: each distinct one is
    // fetched once per thread.
    int2 wp[KF_WPER];
    #pragma unroll
    for (int q = 0; q < KF_WPER; ++q) {
      const bool fresh = q == 0 || widx[q] != widx[q - 1];
      wp[q] = (fresh && widx[q]) ? __ldcg(&sample[widx[q] - 1u]) : make_int2(0, 0);
    }
    #pragma unroll
    for (int q = 1; q < KF_WPER; ++q)
      if (widx[q] == widx[q - 1]) wp[q] = wp[q - 1];
    // Written through the staging area (free until the stream starts) so
    // that consecutive threads write consecutive words: thread t's bins are
    // consecutive, which would put a warp's stores on one bank pair.
    int2* tr = reinterpret_cast<int2*>(&S.key[0][0]);
    static_assert(sizeof(S.key) + sizeof(S.idx) >= sizeof(int2) * KF_WPER * KF_BLOCK &&
                  offsetof(KFSmem, idx) == offsetof(KFSmem, key) + sizeof(S.key), "transpose area");
    #pragma unroll
    for (int q = 0; q < KF_WPER; ++q)
      tr[q * KF_BLOCK + threadIdx.x] = widx[q] ? make_int2(wp[q].x - F.bx, wp[q].y - F.by) : make_int2(F.ux, F.uy);
    __syncthreads();
    for (u32 b = threadIdx.x; b < (u32)kWitnessBins; b += KF_BLOCK)
      S.wt[2 * b + r] = tr[(b % KF_WPER) * KF_BLOCK + b / KF_WPER];
    __syncthreads();      // s_wm and the transpose area are reused by the next region
  }
}

// Strict interior of the block's copy of the filter polygon (fewer than
// three corners: nothing is inside).
__device__ __forceinline__ bool inside_polygon(const KFSmem& S, int x, int y) {
  const int k = S.ncorner;
  bool in = k >= 3;
  for (int j = 0; j < k && in; ++j) {
    const KFEdge e = S.edge[j];
    in = (long long)e.ex * y + (long long)e.ney * x + e.nc > 0;
  }
  return in;
}

// One warp: the staged points [0, fill) of its slice that also survive the
// filter polygon go to the output at one reserved run, their bins' totals
// to btot.
__device__ __noinline__ void warp_flush(const KFSmem& S, u64* skey, u32* sidx, u32 fill, Plan* plan,
                                        const Front& F, u32 cap, u64* __restrict__ okey, u32* __restrict__ oidx,
                                        u32* __restrict__ btot, const u32* __restrict__ imap) {
  const int lane = threadIdx.x & 31;
  constexpr int PER = KF_SLICE / 32;
  __syncwarp();
  bool keep[PER];
  u32 cnt = 0;
  #pragma unroll
  for (int k = 0; k < PER; ++k) {
    const u32 j = lane + 32 * k;
    keep[k] = false;
    if (j < fill) {
      const u64 key = skey[j];
      const int x = F.x0 + (int)(u32)(key >> F.ybits), y = F.y0 + (int)(u32)(key & F.ymask);
      keep[k] = !inside_polygon(S, x, y);
      cnt += keep[k] ? 1u : 0u;
    }
  }
  u32 inc = cnt;
  #pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const u32 t = __shfl_up_sync(0xFFFFFFFFu, inc, o);
    if (lane >= o) inc += t;
  }
  const u32 tot = __shfl_sync(0xFFFFFFFFu, inc, 31);
  u32 base = 0;
  if (lane == 31 && tot) base = atomicAdd(&plan->ctr[CTR_FUSED], tot);
  base = __shfl_sync(0xFFFFFFFFu, base, 31);
  u32 pos = base + inc - cnt;
  #pragma unroll
  for (int k = 0; k < PER; ++k) {
    if (keep[k]) {
      const u32 j = lane + 32 * k;
      const u64 key = skey[j];
      if (pos < cap) {
        okey[pos] = key;
        oidx[pos] = imap ? __ldg(&imap[sidx[j]]) : sidx[j];
        atomicAdd(&btot[(u32)(key >> F.fshift)], 1u);
      } else {
        flag_error(plan, ERR_INTERNAL);
      }
      ++pos;
    }
  }
  __syncwarp();        // the slice is free again
}

// The stream of points of one block (every thread of the block calls it).
template <bool VEC, bool COUNT, bool XONLY>
__device__ __forceinline__ void stream_points(const int* __restrict__ xy, u32 n, Plan* plan, const Front& F, KFSmem& S,
                                              u64* __restrict__ okey, u32* __restrict__ oidx,
                                              u32* __restrict__ btot, const u32* __restrict__ imap, u32* nq_out) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  u64* skey = S.key[wid];
  u32* sidx = S.idx[wid];
  const u32 nt = gridDim.x * KF_BLOCK;
  const u32 kstr = KF_CONTIG ? 32u : nt;   // units between a thread's slots of one round
  u32 fill = 0, nq = 0;
  // Unit j: points 2j and 2j + 1 (an int4 when VEC).  A round takes units
  // j0, j0 + nt, ..., j0 + (KF_V - 1) nt; the rounds whose units all lie
  // below n / 2 need no bounds checks.  In the last round, slots past n take
  // P_l: every slot meets the witness test, whose table index is only in
  // range inside the bounding box.
  const u32 nfull = n / 2;                 // units with both points present
  const u32 nunit = (n + 1) / 2;
  auto load = [&](u32 j0, bool guarded, int4* v) {
    #pragma unroll
    for (int r = 0; r < KF_V; ++r) {
      const u32 j = j0 + r * kstr;
      v[r] = make_int4(F.bx, F.by, F.bx, F.by);
      if (!guarded && VEC) {
        v[r] = reinterpret_cast<const int4*>(xy)[j];
      } else {
        if (2 * j < n) { const int2 a = reinterpret_cast<const int2*>(xy)[2 * j]; v[r].x = a.x; v[r].y = a.y; }
        if (2 * j + 1 < n) { const int2 b = reinterpret_cast<const int2*>(xy)[2 * j + 1]; v[r].z = b.x; v[r].w = b.y; }
      }
    }
  };
  auto round = [&](u32 j0, bool guarded, const int4* v) {
    int px[KF_PTS], py[KF_PTS];
    #pragma unroll
    for (int r = 0; r < KF_V; ++r) {
      px[2 * r] = v[r].x; py[2 * r] = v[r].y; px[2 * r + 1] = v[r].z; py[2 * r + 1] = v[r].w;
    }
    bool pass[KF_PTS];
    u32 cnt = 0;
    #pragma unroll
    for (int e = 0; e < KF_PTS; ++e) {
      const bool in = !guarded || 2u * (j0 + (e >> 1) * kstr) + (u32)(e & 1) < n;
      pass[e] = in && witness_pass<XONLY>(F, S.wt, px[e], py[e]);
      if (COUNT && in) nq += inside_polygon(S, px[e], py[e]) ? 0u : 1u;
      cnt += pass[e] ? 1u : 0u;
    }
    if (__any_sync(0xFFFFFFFFu, cnt != 0)) {
      u32 inc = cnt;
      #pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const u32 t = __shfl_up_sync(0xFFFFFFFFu, inc, o);
        if (lane >= o) inc += t;
      }
      const u32 tot = __shfl_sync(0xFFFFFFFFu, inc, 31);
      if (fill + tot > (u32)KF_SLICE) {            // uniform over the warp
        warp_flush(S, skey, sidx, fill, plan, F, plan->n, okey, oidx, btot, imap);
        fill = 0;
      }
      u32 pos = fill + inc - cnt;
      #pragma unroll
      for (int e = 0; e < KF_PTS; ++e) {
        if (pass[e]) {
          skey[pos] = ((u64)(u32)(px[e] - F.x0) << F.ybits) | (u64)(u32)(py[e] - F.y0);
          sidx[pos] = 2u * (j0 + (e >> 1) * kstr) + (u32)(e & 1);
          ++pos;
        }
      }
      fill += tot;
    }
  };
  // Unit of round 0, slot r: KF_CONTIG gives every warp one contiguous run
  // of 32 KF_V units per round, else slot r of all threads is contiguous.
  u32 j0 = KF_CONTIG ? (blockIdx.x * KF_BLOCK + (threadIdx.x & ~31u)) * KF_V + lane : blockIdx.x * KF_BLOCK + threadIdx.x;
  // Full rounds: every thread of the warp has all KF_V units below nfull
  // (checked on the warp's last lane, so the branch is uniform).
  const u32 lane_last = j0 - lane + 31;
  u32 jl = lane_last;
  if (KF_PF) {
    // The next full round's loads go out before this round is computed.
    int4 cur[KF_V];
    bool have = jl + (KF_V - 1) * kstr < nfull;
    if (have) load(j0, false, cur);
    while (have) {
      const bool more = jl + KF_V * nt + (KF_V - 1) * kstr < nfull;   // uniform over the warp
      int4 nxt[KF_V];
      if (more) load(j0 + KF_V * nt, false, nxt);
      round(j0, false, cur);
      jl += KF_V * nt;
      j0 += KF_V * nt;
      if (more) {
        #pragma unroll
        for (int r = 0; r < KF_V; ++r) cur[r] = nxt[r];
      }
      have = more;
    }
  } else {
    for (; jl + (KF_V - 1) * kstr < nfull; jl += KF_V * nt, j0 += KF_V * nt) {
      int4 v[KF_V];
      load(j0, false, v);
      round(j0, false, v);
    }
  }
  for (; j0 - lane < nunit; j0 += KF_V * nt) {
    int4 v[KF_V];
    load(j0, true, v);
    round(j0, true, v);
  }
  if (fill) warp_flush(S, skey, sidx, fill, plan, F, plan->n, okey, oidx, btot, imap);
  *nq_out = nq;
}

template <bool VEC, bool COUNT>
__global__ void __launch_bounds__(KF_BLOCK, KF_MINB_CFG)
k2_fused(const int* __restrict__ xy, Plan* plan, const u64* __restrict__ wkey, const int2* __restrict__ sample,
         u64* __restrict__ okey, u32* __restrict__ oidx, u32* __restrict__ btot, u32* __restrict__ bstart,
         uint2* __restrict__ groups, u32* __restrict__ fcur, const u32* __restrict__ ncount,
         const u32* __restrict__ imap) {
  extern __shared__ __align__(128) unsigned char kf_smem[];
  KFSmem& S = *reinterpret_cast<KFSmem*>(kf_smem);
  __shared__ u64 s_wm[KF_WARPS];
  __shared__ bool s_last;
  if (plan->error & ERR_RANGE) return;
  // The points: the input (n = plan->n), or the single-read front's raw
  // survivors (n = *ncount, their input indices in imap).
  const u32 n = ncount ? *ncount : plan->n;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const Front F = make_front(plan);
  if (threadIdx.x < kMaxCorners) {
    const int k = plan->ncorner, j = threadIdx.x;
    if (j < k) {
      const int jn = j + 1 < k ? j + 1 : 0;
      const int ax = plan->cx[j], ay = plan->cy[j];
      const int ex = plan->cx[jn] - ax, ey = plan->cy[jn] - ay;
      S.edge[j] = KFEdge{ex, -ey, -((long long)ex * ay - (long long)ey * ax)};
    }
    if (j == 0) S.ncorner = k;
  }
  build_witness_table(wkey, sample, F, S, s_wm);   // its barriers also publish the polygon
  u32 nq = 0;
  if (F.s2 == 0 && F.ysh >= F.ybits)      // uniform: the witness bin depends on x alone
    stream_points<VEC, COUNT, true>(xy, n, plan, F, S, okey, oidx, btot, imap, &nq);
  else
    stream_points<VEC, COUNT, false>(xy, n, plan, F, S, okey, oidx, btot, imap, &nq);
  if (COUNT) {
    #pragma unroll
    for (int o = 16; o > 0; o >>= 1) nq += __shfl_xor_sync(0xFFFFFFFFu, nq, o);
    if (lane == 0 && nq) atomicAdd(&plan->s_quad, nq);
  }
  // The last block turns the bins' totals into bin starts and groups.
  static_assert(sizeof(BinScanSmem) <= sizeof(KFSmem::wt) && KF_BLOCK == BS_BLOCK, "bin scan in the table's place");
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(&plan->ctr[CTR_FUSED_DONE], 1u) == gridDim.x - 1;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  bins_to_groups<true>(btot, plan, bstart, groups, fcur, *reinterpret_cast<BinScanSmem*>(&S.wt[0]));
}

// ---- k2_place: the fused filter's output into coarse-bin order.
constexpr int KP_BLOCK = 256;
constexpr int KP_ITEMS = 8;
constexpr int KP_CHUNK = KP_BLOCK * KP_ITEMS;
constexpr int KP_WARPS = KP_BLOCK / 32;
static_assert(kCoarse == KP_BLOCK, "one thread per coarse bin");
static_assert(KP_CHUNK <= 8192, "rank packed in 13 bits");

__global__ void __launch_bounds__(KP_BLOCK)
k2_place(const u64* __restrict__ ak, const u32* __restrict__ ai, Plan* plan, const u32* __restrict__ bstart,
         u32* __restrict__ ccur, u64* __restrict__ ok, u32* __restrict__ oi) {
  __shared__ u64 s_key[KP_CHUNK];
  __shared__ u32 s_idx[KP_CHUNK];
  __shared__ u32 s_cnt[kCoarse], s_lst[kCoarse], s_gb[kCoarse], s_ws[KP_WARPS];
  if (plan->error & (ERR_RANGE | ERR_FALLBACK)) return;
  const u32 m = plan->s;
  const u32 cshift = plan->fshift + (u32)(kBinBits - kCoarseBits);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (u32 base = blockIdx.x * (u32)KP_CHUNK; base < m; base += gridDim.x * (u32)KP_CHUNK) {
    s_cnt[threadIdx.x] = 0u;
    __syncthreads();
    u64 key[KP_ITEMS];
    u32 idx[KP_ITEMS], rk[KP_ITEMS];
    #pragma unroll
    for (int it = 0; it < KP_ITEMS; ++it) {
      const u32 i = base + it * KP_BLOCK + threadIdx.x;
      key[it] = i < m ? ak[i] : 0ull;
      idx[it] = i < m ? ai[i] : 0u;
    }
    #pragma unroll
    for (int it = 0; it < KP_ITEMS; ++it) {
      const u32 i = base + it * KP_BLOCK + threadIdx.x;
      rk[it] = i < m ? atomicAdd(&s_cnt[(u32)(key[it] >> cshift)], 1u) : 0xFFFFFFFFu;
    }
    __syncthreads();
    {
      const u32 cb = threadIdx.x;
      const u32 cn = s_cnt[cb];
      u32 inc = cn;
      #pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const u32 t = __shfl_up_sync(0xFFFFFFFFu, inc, o);
        if (lane >= o) inc += t;
      }
      if (lane == 31) s_ws[wid] = inc;
      s_gb[cb] = cn ? bstart[cb * kFinePerCoarse] + atomicAdd(&ccur[cb], cn) : 0u;
      __syncthreads();
      u32 off = inc - cn;
      for (int w = 0; w < wid; ++w) off += s_ws[w];
      s_lst[cb] = off;
    }
    __syncthreads();
    #pragma unroll
    for (int it = 0; it < KP_ITEMS; ++it) {
      if (rk[it] != 0xFFFFFFFFu) {
        const u32 p = s_lst[(u32)(key[it] >> cshift)] + rk[it];
        s_key[p] = key[it];
        s_idx[p] = idx[it];
      }
    }
    __syncthreads();
    const u32 total = min(m - base, (u32)KP_CHUNK);
    for (u32 j = threadIdx.x; j < total; j += KP_BLOCK) {
      const u64 k = s_key[j];
      const u32 cb = (u32)(k >> cshift);
      const u32 pos = s_gb[cb] + (j - s_lst[cb]);
      if (pos < m) {
        ok[pos] = k;
        oi[pos] = s_idx[j];
      } else {
        flag_error(plan, ERR_INTERNAL);
      }
    }
    __syncthreads();
  }
}

}  // namespace

cudaError_t fused_configure() {
  cudaError_t e = cudaSuccess;
  for (const void* f : {(const void*)k2_fused<true, false>, (const void*)k2_fused<true, true>,
                        (const void*)k2_fused<false, false>, (const void*)k2_fused<false, true>})
    if (e == cudaSuccess) e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)KF_SMEM);
  return e;
}

cudaError_t fused_occupancy(int* blocks) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, k2_fused<true, false>, KF_BLOCK, KF_SMEM);
}

cudaError_t launch_witness(const int2* sample, u32 n, Plan* plan, u64* wkey, int num_sms, cudaStream_t st,
                           const u32* ncount) {
  const u32 samples = ncount ? n : (n + kSampleStride - 1) / kSampleStride;   // a bound with ncount
  u32 grid = (samples + SW_BLOCK * SW_ITEMS - 1) / (SW_BLOCK * SW_ITEMS);   // one round per thread
  const u32 cap = (u32)num_sms * 4u;
  grid = grid < 1 ? 1 : (grid > cap ? cap : grid);
  k_witness<<<grid, SW_BLOCK, 0, st>>>(sample, plan, wkey, ncount);
  return cudaGetLastError();
}

cudaError_t launch_k2_fused(const int* xy, u32 n, Plan* plan, const u64* wkey, const int2* sample, u64* okey,
                            u32* oidx, u32* btot, u32* bstart, uint2* groups, u32* fcur, bool count, int grid,
                            cudaStream_t st, const u32* ncount, const u32* imap) {
  const bool vec = (reinterpret_cast<uintptr_t>(xy) & 15u) == 0;
  const u32 rounds = ((n + 1) / 2 + KF_BLOCK * KF_V - 1) / (KF_BLOCK * KF_V);   // blocks with a full round
  if ((u32)grid > rounds) grid = (int)(rounds < 1 ? 1 : rounds);
  if (vec) {
    if (count) k2_fused<true, true><<<grid, KF_BLOCK, KF_SMEM, st>>>(xy, plan, wkey, sample, okey, oidx, btot, bstart, groups, fcur, ncount, imap);
    else k2_fused<true, false><<<grid, KF_BLOCK, KF_SMEM, st>>>(xy, plan, wkey, sample, okey, oidx, btot, bstart, groups, fcur, ncount, imap);
  } else {
    if (count) k2_fused<false, true><<<grid, KF_BLOCK, KF_SMEM, st>>>(xy, plan, wkey, sample, okey, oidx, btot, bstart, groups, fcur, ncount, imap);
    else k2_fused<false, false><<<grid, KF_BLOCK, KF_SMEM, st>>>(xy, plan, wkey, sample, okey, oidx, btot, bstart, groups, fcur, ncount, imap);
  }
  return cudaGetLastError();
}

cudaError_t launch_place(const u64* ak, const u32* ai, u32 n, Plan* plan, const u32* bstart, u32* ccur, u64* ok,
                         u32* oi, int num_sms, cudaStream_t st) {
  const u32 chunks = (n + KP_CHUNK - 1) / KP_CHUNK;
  const u32 cap = (u32)num_sms * 4u;
  const u32 grid = chunks < 1 ? 1u : (chunks > cap ? cap : chunks);
  k2_place<<<grid, KP_BLOCK, 0, st>>>(ak, ai, plan, bstart, ccur, ok, oi);
  return cudaGetLastError();
}

}  // namespace gbh
