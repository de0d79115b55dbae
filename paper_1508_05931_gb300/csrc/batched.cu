// Batched hulls: many independent point sets in one call.
//
// k_batch, mode 0: every block takes instances from a queue ordered largest
// first (so the longest jobs start early and the small ones fill the tail)
// and runs the whole pipeline of Section 2.1 on one instance by itself, each
// step as a block-level loop over chunks in order, so no block ever waits
// for another:
//   1. extremes (step 1): block reduction, every 32nd point copied out;
//   1b. witnesses: every sampled point that survives the filter polygon is
//      a witness for every later witness bin of its region; the block keeps
//      each bin's most advanced one and turns them into every bin's
//      exclusive prefix (as the single-hull front does, k2_fused.cu: a point
//      not strictly beyond a first-round survivor before it is one Figure 2
//      discards, so the second round's result is unchanged);
//   2. the witness test, then the filter polygon (steps 2-3) on the witness
//      survivors staged per warp, compaction in input order, survivors
//      counted per witness bin;
//   3. the sort (step 4) by (key, index): survivors moved into shared
//      memory by witness bin and every bin sorted there (by rank, or by the
//      block's bitonic network), in groups of bins when they do not fit at
//      once; a stable LSD radix sort through the scratch region when one
//      bin alone does not fit;
//   4. region split + second round (steps 5-7) as a running prefix
//      max/min of directions seen from P_l (exactly Figure 2's survivors);
//   5. lower and upper chains (step 8): chunks of the chain built in shared
//      memory (per-thread stacks, warp bridge merges), then chunk chains
//      merged level by level through global scratch.
// The segmented path of the largest instances splits this: k_seg_ext
// (step 1, flat over all their tiles), k_batch mode 1 (the plan and step
// 1b per instance), k_seg_filter (step 2, flat over the tiles) and k_batch
// mode 2 (the survivors gathered, then steps 3-5 per instance).
// Each instance owns a scratch region of its size plus a fixed pad; its
// hull (CCW indices relative to the instance) is staged there and a second
// kernel compacts all hulls into the output with their offsets.
#include "chain.cuh"
#include "hull_internal.cuh"
#include "kernels.h"
#include "learned_common.cuh"

namespace gbh {

using namespace chain;

namespace {

constexpr int BT_ITEMS = 16;        // sort keys per thread per tile
constexpr int BT_FITEMS = 8;        // filter / second-round items per thread per chunk
constexpr int BT_LEAF = 8;          // chain points per thread
constexpr int BT_MAX_CHUNKS = 1024; // chain chunks per instance (bounds n_i)
constexpr int BW_BITS = 9;          // witness bins per instance: the top BW_BITS of the key
constexpr int BW_BINS = 1 << BW_BITS;
constexpr u32 BW_STRIDE = 32;       // one sampled point in every BW_STRIDE
constexpr u32 BT_RANKMAX = 64;      // witness bins up to this size are sorted by rank, larger ones by the block
constexpr u32 BL_MIN_N = 262144;    // smallest instance the learned proposal runs on

struct BestX {
  u64 k[4];
  u32 i[4];
};

__device__ __forceinline__ void bx_init(BestX& b) {
  #pragma unroll
  for (int j = 0; j < 4; ++j) { b.k[j] = ~0ull; b.i[j] = 0xFFFFFFFFu; }
}
__device__ __forceinline__ bool bx_lt(u64 ka, u32 ia, u64 kb, u32 ib) {
  return ka < kb || (ka == kb && ia < ib);
}
__device__ __forceinline__ void bx_point(BestX& b, int x, int y, u32 idx) {
  const u32 ox = (u32)x ^ 0x80000000u, oy = (u32)y ^ 0x80000000u;
  const u64 kxy = ((u64)ox << 32) | oy, kyx = ((u64)oy << 32) | ox;
  if (kxy < b.k[0]) { b.k[0] = kxy; b.i[0] = idx; }
  if (~kxy < b.k[1]) { b.k[1] = ~kxy; b.i[1] = idx; }
  if (kyx < b.k[2]) { b.k[2] = kyx; b.i[2] = idx; }
  if (~kyx < b.k[3]) { b.k[3] = ~kyx; b.i[3] = idx; }
}
__device__ __forceinline__ void bx_merge(BestX& a, const u64* k, const u32* i) {
  #pragma unroll
  for (int j = 0; j < 4; ++j)
    if (bx_lt(k[j], i[j], a.k[j], a.i[j])) { a.k[j] = k[j]; a.i[j] = i[j]; }
}
__device__ __forceinline__ void bx_warp(BestX& b) {
  #pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    u64 k[4]; u32 i[4];
    #pragma unroll
    for (int j = 0; j < 4; ++j) {
      k[j] = __shfl_xor_sync(0xFFFFFFFFu, b.k[j], o);
      i[j] = __shfl_xor_sync(0xFFFFFFFFu, b.i[j], o);
    }
    bx_merge(b, k, i);
  }
}

__device__ __forceinline__ u32 bitlen32(u32 v) { return v ? 32u - (u32)__clz(v) : 0u; }

// Strictly inside the filter polygon (k >= 3 edges in shared memory, each
// {e_x, -e_y, low and high words of the constant}: the edge's cross product
// with the point, positive strictly inside).
__device__ __forceinline__ bool in_polygon(const int4* E, int k, int x, int y) {
  bool in = k >= 3;
  for (int e = 0; e < k && in; ++e) {
    const int4 q = E[e];
    const long long c = (long long)(((u64)(u32)q.w << 32) | (u64)(u32)q.z);
    in = (long long)q.x * y + (long long)q.y * x + c > 0;
  }
  return in;
}

// Per-instance parameters, built by thread 0 from the extremes.
struct IPlan {
  int ext_idx[4];
  int ext_x[4], ext_y[4];
  int ncorner;
  int learned;
  int x0, y0;
  u32 ybits, npasses;
  u32 kbits;
  int bad;
};

// Sorting (key, index) pairs in shared memory; pairs are distinct because
// the indices are.
__device__ __forceinline__ bool pair_lt(u64 ka, u32 va, u64 kb, u32 vb) {
  return ka < kb || (ka == kb && va < vb);
}
__device__ __forceinline__ void pair_ce(u64* K, u32* V, u32 i, u32 l) {
  const u64 ki = K[i], kl = K[l];
  const u32 vi = V[i], vl = V[l];
  if (pair_lt(kl, vl, ki, vi)) { K[i] = kl; K[l] = ki; V[i] = vl; V[l] = vi; }
}
// Bitonic network of the next power of two N >= m in its form without
// direction flags (the first step of every merge compares an element with
// its mirror in the merged block, the rest are half-cleaners, every
// compare-exchange puts the smaller pair first).  The slots past m hold an
// implicit maximum that no compare-exchange would move, so exchanges that
// reach past m are skipped.  Lanes [0, nthr) of the calling group (warp or
// block) take the pairs of every step; sync() separates the steps.
template <typename Sync>
__device__ __forceinline__ void bitonic_pairs(u64* K, u32* V, u32 m, u32 t0, u32 nthr, Sync sync) {
  u32 N = 1;
  while (N < m) N <<= 1;
  for (u32 k = 2; k <= N; k <<= 1) {
    for (u32 j = k >> 1; j > 0; j >>= 1) {
      const u32 lj = (u32)__ffs(j) - 1u;
      for (u32 t = t0; t < N / 2; t += nthr) {
        const u32 g = t >> lj, o = t & (j - 1u);
        u32 i, l;
        if (j == k >> 1) { i = g * k + o; l = g * k + k - 1u - o; }
        else { i = g * 2u * j + o; l = i + j; }
        if (l < m) pair_ce(K, V, i, l);
      }
      sync();
    }
  }
}
struct Dir2b {
  int lx, ly, ux, uy;
};
__device__ __forceinline__ void dcombine(Dir2b& a, const Dir2b& b) {
  bool t = cross2(a.lx, a.ly, b.lx, b.ly) > 0;
  a.lx = t ? b.lx : a.lx; a.ly = t ? b.ly : a.ly;
  t = cross2(a.ux, a.uy, b.ux, b.uy) < 0;
  a.ux = t ? b.ux : a.ux; a.uy = t ? b.uy : a.uy;
}
__device__ __forceinline__ Dir2b dshfl_up(const Dir2b& v, int o) {
  Dir2b r;
  r.lx = __shfl_up_sync(0xFFFFFFFFu, v.lx, o); r.ly = __shfl_up_sync(0xFFFFFFFFu, v.ly, o);
  r.ux = __shfl_up_sync(0xFFFFFFFFu, v.ux, o); r.uy = __shfl_up_sync(0xFFFFFFFFu, v.uy, o);
  return r;
}

template <int BLOCK>
struct Smem {
  static constexpr int W = BLOCK / 32;
  static constexpr int CHUNK = BLOCK * BT_LEAF;   // chain points per shared-memory chunk
  static constexpr int SCAP = BLOCK == 512 ? 14336 : 6144;   // survivors sorted in shared memory
  u32 wpos[W][kRadix];
  u32 hist[kMaxPasses][kRadix];
  u32 cur[kRadix];
  u32 red[BT_FITEMS * W + 8];
  Dir2b wdir[W];
  u32 wcnt[W][2];
  IPlan plan;
  int inst;
  int hq;                            // position of the instance in `order`
  u64 rk[W][4];
  u32 ri[W][4];
  union {
    struct {                         // chains (step 5)
      int sx[CHUNK], sy[CHUNK], si[CHUNK];
    };
    struct {                         // learned proposal (step 1)
      learned::FeatSmem feat;
      learned::MlpSmem mlp;
      int ext_xy[2 * learned::NB];
      int ext_idx[learned::NB];
    };
    struct {                         // witnesses (steps 1b-2)
      int2 wtab[2 * BW_BINS];        // witness direction of (bin, region)
      union {
        u64 wkey[2 * BW_BINS];       // step 1b: the sample's best witness per (region, bin)
        struct {                     // step 2: every warp's witness survivors of a round
          int2 sxy[W][32 * BT_FITEMS];
          u32 sidx[W][32 * BT_FITEMS];
        } st;
      };
    };
    struct {                         // sort by bins (steps 3-4)
      u64 bk[SCAP];
      u32 bi[SCAP];
    };
  };
  u64 wmax[W];
  int ccnt[BLOCK];                   // per-thread chain lengths inside a chunk
  int corner_x[kMaxCorners + 4], corner_y[kMaxCorners + 4];
  int4 edge[kMaxCorners];            // the filter polygon's edges (in_polygon)
  u32 nbig;                          // witness bins above BT_RANKMAX survivors
  unsigned short bigl[BW_BINS];      // those bins
  u32 ngrp;                          // groups of bins sorted one at a time (more than SCAP survivors)
  int bbox[4];                       // the skip box of step 1
  unsigned short big[BW_BINS];
  int chunk_cnt[BT_MAX_CHUNKS];      // chain length of every chunk
  int4 pair[BT_MAX_CHUNKS / 2];      // bridge results of one merge level
};

// The learned proposal's fixed cost (features of a 4,096-point sample and
// the MLP) is paid only by instances of at least BL_MIN_N points whose
// quadrilateral leaves more than 5 % of a strided 512-point sample (the gate
// of the single-hull proposal).  Past the gate: features of a sample of the
// instance, the MLP, the exact hull of the quadrilateral and the 8 chosen
// extremes.  Kept out of line: it runs once per instance and its locals
// would crowd the streaming loops' registers.
template <int BLOCK>
__device__ __noinline__ void learned_step(Smem<BLOCK>& S, const int2* P, u32 n, const __half* w16) {
  if (threadIdx.x == 0) S.nbig = 0;
  __syncthreads();
  if (S.plan.ncorner >= 3) {
    constexpr u32 G = 512;
    for (u32 t = threadIdx.x; t < G; t += BLOCK) {
      const int2 q = P[(u32)(((unsigned long long)t * n) / G)];
      bool in = true;
      for (int j = 0; j < S.plan.ncorner && in; ++j) {
        const int jn = j + 1 < S.plan.ncorner ? j + 1 : 0;
        in = orient(S.corner_x[j], S.corner_y[j], S.corner_x[jn], S.corner_y[jn], q.x, q.y) > 0;
      }
      if (in) atomicAdd(&S.nbig, 1u);
    }
  }
  __syncthreads();
  if (S.nbig >= 487u) return;   // 487 / 512 > 95 %
  const u32 smp = n < 4096u ? n : 4096u;
  learned::block_features<BLOCK>(P, n, smp, S.feat, S.mlp.x, S.ext_xy, S.ext_idx);
  learned::block_mlp(w16, S.mlp);
  if (threadIdx.x == 0) {
    int qx[4], qy[4], ox[kMaxCorners], oy[kMaxCorners];
    const int nq = S.plan.ncorner < 4 ? S.plan.ncorner : 4;
    for (int j = 0; j < nq; ++j) { qx[j] = S.corner_x[j]; qy[j] = S.corner_y[j]; }
    const int k2 = learned::learned_polygon(S.mlp.z, S.ext_xy, qx, qy, nq, ox, oy);
    if (k2 > 0) {
      S.plan.ncorner = k2;
      S.plan.learned = 1;
      for (int j = 0; j < k2; ++j) { S.corner_x[j] = ox[j]; S.corner_y[j] = oy[j]; }
    }
  }
  __syncthreads();
}

// Sorts the pairs of bins [g0, g1) staged in shared memory (S.bk / S.bi
// [0, m): the bins in order, bin b at [bend[b] - bcnt[b] - p0, bend[b] -
// p0), its pairs in any order) by (key, index) into dk / di [p0, p0 + m).
// A pair of a bin of at most BT_RANKMAX pairs goes straight to its place:
// its bin's start plus the number of the bin's pairs below it (pairs are
// distinct: the indices are).  Larger bins are sorted in place by the whole
// block's bitonic network, one at a time, and copied out.
template <int BLOCK>
__device__ void sort_bins_out(Smem<BLOCK>& S, const u32* bcnt, const u32* bend, u32 g0, u32 g1, u32 p0, u32 m,
                              u32 wshift, u64* dk, u32* di) {
  if (threadIdx.x == 0) S.nbig = 0;
  __syncthreads();
  for (u32 b = g0 + threadIdx.x; b < g1; b += BLOCK)
    if (bcnt[b] > BT_RANKMAX) S.bigl[atomicAdd(&S.nbig, 1u)] = (unsigned short)b;
  for (u32 i = threadIdx.x; i < m; i += BLOCK) {
    const u64 k = S.bk[i];
    const u32 v = S.bi[i];
    const u32 b = (u32)(k >> wshift);
    const u32 c = bcnt[b];
    if (c > BT_RANKMAX) continue;
    const u32 b0 = bend[b] - c - p0;
    u32 r = 0;
    for (u32 j = b0; j < b0 + c; ++j) r += pair_lt(S.bk[j], S.bi[j], k, v) ? 1u : 0u;
    dk[p0 + b0 + r] = k;
    di[p0 + b0 + r] = v;
  }
  __syncthreads();
  const u32 nb = S.nbig;
  for (u32 q = 0; q < nb; ++q) {
    const u32 b = S.bigl[q], c = bcnt[b], b0 = bend[b] - c - p0;
    bitonic_pairs(S.bk + b0, S.bi + b0, c, threadIdx.x, (u32)BLOCK, [] { __syncthreads(); });
    for (u32 i = threadIdx.x; i < c; i += BLOCK) {
      dk[p0 + b0 + i] = S.bk[b0 + i];
      di[p0 + b0 + i] = S.bi[b0 + i];
    }
  }
  __syncthreads();
}

// Chain over m points (xy, idx) in lexicographic order.  Short chains are
// built in shared memory and left there; longer ones are built in chunks
// and merged through g0/g1.  Returns the chain length; *where receives 0
// (shared memory), 1 (g0) or 2 (g1).
template <int BLOCK>
__device__ int build_chain(Smem<BLOCK>& S, const int2* xy, const int* idx, int m, int sgn,
                           int2* g0xy, int* g0i, int2* g1xy, int* g1i, int* where) {
  constexpr int CHUNK = Smem<BLOCK>::CHUNK;
  constexpr int W = Smem<BLOCK>::W;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nch = (m + CHUNK - 1) / CHUNK;
  for (int ch = 0; ch < nch; ++ch) {
    const int first = ch * CHUNK;
    const int len = min(CHUNK, m - first);
    for (int i = threadIdx.x; i < len; i += BLOCK) {
      const int2 p = xy[first + i];
      S.sx[i] = p.x; S.sy[i] = p.y; S.si[i] = idx[first + i];
    }
    __syncthreads();
    const int b = threadIdx.x * BT_LEAF;
    S.ccnt[threadIdx.x] = leaf_chain(S.sx, S.sy, S.si, b, max(0, min(BT_LEAF, len - b)), sgn);
    __syncthreads();
    const int nleaf = (len + BT_LEAF - 1) / BT_LEAF;
    merge_tree<BT_LEAF>(S.sx, S.sy, S.si, S.ccnt, S.pair, nleaf, sgn);
    const int hc = S.ccnt[0];
    if (nch == 1) { *where = 0; return hc; }
    for (int i = threadIdx.x; i < hc; i += BLOCK) {
      g0xy[first + i] = make_int2(S.sx[i], S.sy[i]);
      g0i[first + i] = S.si[i];
    }
    if (threadIdx.x == 0) S.chunk_cnt[ch] = hc;
    __syncthreads();
  }
  // Merge chunk chains level by level (ping-pong through g0 / g1).
  int2* cx = g0xy; int* ci = g0i; int2* nx = g1xy; int* ni = g1i;
  int buf = 1;
  for (int step = 1; step < nch; step <<= 1) {
    const int np = (nch + 2 * step - 1) / (2 * step);
    for (int p = wid; p < np; p += W) {
      const int ca = 2 * p * step, cb = ca + step;
      const int alpha = S.chunk_cnt[ca];
      int is = alpha - 1, js = 0, beta = 0;
      if (cb < nch) {
        beta = S.chunk_cnt[cb];
        GlobalChain A{cx + (size_t)ca * CHUNK}, Bc{cx + (size_t)cb * CHUNK};
        bridge(A, alpha, Bc, beta, sgn, is, js);
      }
      if (lane == 0) S.pair[p] = make_int4(is, js, beta, 0);
    }
    __syncthreads();
    for (int p = 0; p < np; ++p) {
      const int4 pr = S.pair[p];
      const int merged = pr.x + 1 + (pr.z - pr.y);
      const size_t abase = (size_t)(2 * p * step) * CHUNK;
      const size_t bbase = abase + (size_t)step * CHUNK;
      for (int o = threadIdx.x; o < merged; o += BLOCK) {
        const size_t src = (o <= pr.x) ? abase + o : bbase + pr.y + (o - pr.x - 1);
        nx[abase + o] = __ldcg(&cx[src]);
        ni[abase + o] = __ldcg(&ci[src]);
      }
    }
    __syncthreads();
    for (int p = threadIdx.x; p < np; p += BLOCK) {
      const int4 pr = S.pair[p];
      S.chunk_cnt[2 * p * step] = pr.x + 1 + (pr.z - pr.y);
    }
    __syncthreads();
    int2* t0 = cx; cx = nx; nx = t0;
    int* t1 = ci; ci = ni; ni = t1;
    buf ^= 1;
  }
  *where = buf == 1 ? 1 : 2;
  return S.chunk_cnt[0];
}

// The segmented path (instances of batch_seg_min() points or more): the
// extremes of every tile run, and every instance's record for the second
// streaming pass and the gather.
constexpr u32 SEG_TILE = 16384;     // points per tile (a multiple of 512 x BT_FITEMS)
struct SegTileExt {
  u64 k[4];
  u32 i[4];
};
struct SegRec {
  IPlan plan;
  int4 edge[kMaxCorners];
  int2 wtab[2 * BW_BINS];
};

struct BatchArgs {
  const int* xy;
  const long long* offsets;   // [B + 1]
  const int* order;           // instances of this launch, largest first
  int nb;
  u32* queue;
  const long long* slot0;     // [B] scratch region of each instance
  u64* ka; u64* kb; u32* ia; u32* ib;
  int2* lxy; int* lidx; int2* uxy; int* uidx;
  int* out_tmp;
  u32* hcount;                // [B]
  u32* error;
  const __half* w16;          // learned proposal weights (null: quadrilateral)
  int mode;                   // 0 whole pipeline, 1 plan + witnesses from tiles, 2 gather + back half
  const int* tfirst;          // [nb + 1] first tile of every instance of `order` (modes 1, 2)
  SegTileExt* text;
  u32* tcnt;
  SegRec* rec;                // [nb], indexed like `order`
};

template <int BLOCK, int MODE>
__global__ void __launch_bounds__(BLOCK)
k_batch(BatchArgs a) {
  extern __shared__ __align__(16) unsigned char bt_smem[];
  Smem<BLOCK>& S = *reinterpret_cast<Smem<BLOCK>*>(bt_smem);
  constexpr int W = Smem<BLOCK>::W;
  constexpr int TILE = BLOCK * BT_ITEMS;
  constexpr int FCH = BLOCK * BT_FITEMS;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const u32 lt_mask = (1u << lane) - 1u;

  for (;;) {
    if (threadIdx.x == 0) {
      const u32 q = atomicAdd(a.queue, 1u);
      S.inst = q < (u32)a.nb ? a.order[q] : -1;
      S.hq = (int)q;
    }
    __syncthreads();
    const int inst = S.inst;
    if (inst < 0) break;
    const long long off = a.offsets[inst];
    const u32 n = (u32)(a.offsets[inst + 1] - off);
    const long long sl = a.slot0[inst];
    const int2* P = reinterpret_cast<const int2*>(a.xy) + off;
    if (n == 0) {
      if (threadIdx.x == 0) a.hcount[inst] = 0;
      __syncthreads();
      continue;
    }

    // ---- 1. extremes (every BW_STRIDE-th point copied to the sort's second
    // key buffer, free until step 3, for the witnesses)
    // (BT_FITEMS points per thread and round, loaded before any is used).
    // The skip box is the bounding box of the first round's points: a point
    // strictly inside a box spanned by input points is no extreme, so only
    // the points on or outside it go through the extreme updates.
    int2* smp = reinterpret_cast<int2*>(a.kb + sl);
    if (MODE == 2) {
      // The plan, polygon and witnesses were built by mode 1 and used by
      // k_seg_filter; only the plan is needed from here on.
      if (threadIdx.x == 0) S.plan = a.rec[S.hq].plan;
      for (int q = threadIdx.x; q < kMaxPasses * kRadix; q += BLOCK) (&S.hist[0][0])[q] = 0u;
      __syncthreads();
    } else {
    BestX b;
    bx_init(b);
    if (MODE == 1) {
      // The tile runs' extremes from k_seg_ext.
      const int tf = a.tfirst[S.hq], te = a.tfirst[S.hq + 1];
      for (int t = tf + (int)threadIdx.x; t < te; t += BLOCK) bx_merge(b, a.text[t].k, a.text[t].i);
    } else {
    if (threadIdx.x == 0) {
      S.bbox[0] = 0x7FFFFFFF; S.bbox[1] = (int)0x80000000; S.bbox[2] = 0x7FFFFFFF; S.bbox[3] = (int)0x80000000;
    }
    __syncthreads();
    {
      int x0 = 0x7FFFFFFF, x1 = (int)0x80000000, y0 = 0x7FFFFFFF, y1 = (int)0x80000000;
      #pragma unroll
      for (int r = 0; r < BT_FITEMS; ++r) {
        const u32 j = r * BLOCK + threadIdx.x;
        if (j < n) {
          const int2 q = P[j];
          x0 = min(x0, q.x); x1 = max(x1, q.x); y0 = min(y0, q.y); y1 = max(y1, q.y);
        }
      }
      #pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        x0 = min(x0, __shfl_xor_sync(0xFFFFFFFFu, x0, o)); x1 = max(x1, __shfl_xor_sync(0xFFFFFFFFu, x1, o));
        y0 = min(y0, __shfl_xor_sync(0xFFFFFFFFu, y0, o)); y1 = max(y1, __shfl_xor_sync(0xFFFFFFFFu, y1, o));
      }
      if (lane == 0 && x0 <= x1) {
        atomicMin(&S.bbox[0], x0); atomicMax(&S.bbox[1], x1); atomicMin(&S.bbox[2], y0); atomicMax(&S.bbox[3], y1);
      }
    }
    __syncthreads();
    const int kx0 = S.bbox[0], kx1 = S.bbox[1], ky0 = S.bbox[2], ky1 = S.bbox[3];
    // The next round's points are loaded before this round's are used.
    int2 p[BT_FITEMS];
    #pragma unroll
    for (int r = 0; r < BT_FITEMS; ++r) {
      const u32 j = r * BLOCK + threadIdx.x;
      p[r] = j < n ? P[j] : make_int2(0, 0);
    }
    for (u32 base = 0; base < n; base += FCH) {
      int2 q[BT_FITEMS];
      #pragma unroll
      for (int r = 0; r < BT_FITEMS; ++r) {
        const u32 j = base + FCH + r * BLOCK + threadIdx.x;
        q[r] = j < n ? P[j] : make_int2(0, 0);
      }
      #pragma unroll
      for (int r = 0; r < BT_FITEMS; ++r) {
        const u32 j = base + r * BLOCK + threadIdx.x;
        if (j < n) {
          if (!(p[r].x > kx0 && p[r].x < kx1 && p[r].y > ky0 && p[r].y < ky1)) bx_point(b, p[r].x, p[r].y, j);
          if (j % BW_STRIDE == 0) smp[j / BW_STRIDE] = p[r];
        }
      }
      #pragma unroll
      for (int r = 0; r < BT_FITEMS; ++r) p[r] = q[r];
    }
    }   // mode 0
    bx_warp(b);
    if (lane == 0)
      for (int q = 0; q < 4; ++q) { S.rk[wid][q] = b.k[q]; S.ri[wid][q] = b.i[q]; }
    __syncthreads();
    if (threadIdx.x == 0) {
      bx_init(b);
      for (int w = 0; w < W; ++w) bx_merge(b, S.rk[w], S.ri[w]);
      IPlan& pl = S.plan;
      int ex[4], ey[4];
      ex[0] = (int)(u32)((b.k[0] >> 32) ^ 0x80000000u); ey[0] = (int)((u32)b.k[0] ^ 0x80000000u);
      u64 k1 = ~b.k[1];
      ex[1] = (int)(u32)((k1 >> 32) ^ 0x80000000u); ey[1] = (int)((u32)k1 ^ 0x80000000u);
      ey[2] = (int)(u32)((b.k[2] >> 32) ^ 0x80000000u); ex[2] = (int)((u32)b.k[2] ^ 0x80000000u);
      u64 k3 = ~b.k[3];
      ey[3] = (int)(u32)((k3 >> 32) ^ 0x80000000u); ex[3] = (int)((u32)k3 ^ 0x80000000u);
      for (int j = 0; j < 4; ++j) { pl.ext_idx[j] = (int)b.i[j]; pl.ext_x[j] = ex[j]; pl.ext_y[j] = ey[j]; }
      pl.bad = (ex[0] < -kCoordLimit || ex[1] > kCoordLimit || ey[2] < -kCoordLimit || ey[3] > kCoordLimit);
      const int ord[4] = {0, 2, 1, 3};
      int k = 0, cx[4], cy[4];
      for (int j = 0; j < 4; ++j) {
        const int x = ex[ord[j]], y = ey[ord[j]];
        if (k > 0 && cx[k - 1] == x && cy[k - 1] == y) continue;
        cx[k] = x; cy[k] = y; ++k;
      }
      while (k > 1 && cx[k - 1] == cx[0] && cy[k - 1] == cy[0]) --k;
      pl.ncorner = k;
      pl.learned = 0;
      for (int j = 0; j < k; ++j) { S.corner_x[j] = cx[j]; S.corner_y[j] = cy[j]; }
      pl.x0 = ex[0]; pl.y0 = ey[2];
      const u32 yb = bitlen32((u32)(ey[3] - ey[2])), xb = bitlen32((u32)(ex[1] - ex[0]));
      pl.ybits = yb;
      pl.kbits = xb + yb;
      pl.npasses = (xb + yb + kRadixBits - 1) / kRadixBits;
      if (pl.bad) atomicOr(a.error, ERR_RANGE);
    }
    __syncthreads();
    if (a.w16 != nullptr && !S.plan.bad && n >= BL_MIN_N) learned_step<BLOCK>(S, P, n, a.w16);
    if (threadIdx.x == 0) {
      IPlan& pl = S.plan;
      const int k = pl.ncorner;
      for (int j = 0; j < kMaxCorners; ++j) {
        const int jj = j < k ? j : 0, jn = (j + 1 < k) ? j + 1 : 0;
        const int e_x = S.corner_x[jn] - S.corner_x[jj], e_y = S.corner_y[jn] - S.corner_y[jj];
        const long long c = -((long long)e_x * S.corner_y[jj] - (long long)e_y * S.corner_x[jj]);
        S.edge[j] = make_int4(e_x, -e_y, (int)(u32)(u64)c, (int)(u32)((u64)c >> 32));
      }
    }
    for (int q = threadIdx.x; q < kMaxPasses * kRadix; q += BLOCK) (&S.hist[0][0])[q] = 0u;
    __syncthreads();
    }   // modes 0, 1
    if (S.plan.bad) {
      if (threadIdx.x == 0) {
        a.hcount[inst] = 0;
        if (MODE == 1) a.rec[S.hq].plan = S.plan;
      }
      __syncthreads();
      continue;
    }
    // The plan's scalars in registers (nothing indexed at run time: no
    // local-memory copy); the polygon's edges stay in shared memory.
    const int ax = S.plan.ext_x[0], ay = S.plan.ext_y[0], bxp = S.plan.ext_x[1], byp = S.plan.ext_y[1];
    const int ext0 = S.plan.ext_idx[0], ext1 = S.plan.ext_idx[1];
    const int x0 = S.plan.x0, y0 = S.plan.y0, ncorner = S.plan.ncorner;
    const u32 ybits = S.plan.ybits, npasses = S.plan.npasses, kbits = S.plan.kbits;

    // ---- 1b. witnesses of the sampled first-round survivors
    const int ux = bxp - ax, uy = byp - ay, d0x = ax - bxp, d0y = ay - byp;
    const u32 wshift = kbits > (u32)BW_BITS ? kbits - (u32)BW_BITS : 0u;
    // The witness bin key >> wshift in 32-bit words: x's bits alone when the
    // shift drops all of y's, else x's shifted up beside y's top bits.
    const bool wx_only = wshift >= ybits;
    const u32 wsx = wx_only ? wshift - ybits : ybits - wshift;
    if (MODE != 2) {
    for (int q = threadIdx.x; q < 2 * BW_BINS; q += BLOCK) S.wkey[q] = 0ull;
    __syncthreads();
    {
      const u32 ns = (n + BW_STRIDE - 1) / BW_STRIDE;
      for (u32 i0 = 0; i0 < ns; i0 += FCH) {
      int2 sp[BT_FITEMS];
      #pragma unroll
      for (int r = 0; r < BT_FITEMS; ++r) {
        const u32 i = i0 + r * BLOCK + threadIdx.x;
        sp[r] = i < ns ? __ldcg(&smp[i]) : make_int2(0, 0);
      }
      #pragma unroll
      for (int r = 0; r < BT_FITEMS; ++r) {
        const u32 i = i0 + r * BLOCK + threadIdx.x;
        if (i >= ns) continue;
        const int2 p = sp[r];
        if (in_polygon(S.edge, ncorner, p.x, p.y)) continue;    // not a first-round survivor
        const int dx = p.x - bxp, dy = p.y - byp;
        const long long c = cross2(d0x, d0y, dx, dy);            // > 0 lower, < 0 upper
        if (c == 0) continue;
        const long long e2 = (long long)d0x * dx + (long long)d0y * dy;
        const float fc = fabsf((float)c), fe = (float)e2;
        const float qa = 1.0f - fe / (fabsf(fe) + fc);           // monotone pseudo-angle from P_0 - P_l
        const u32 quant = (u32)fminf(fmaxf(qa, 0.0f) * 2147483648.0f, 4294967040.0f);
        const u64 key = ((u64)(u32)(p.x - x0) << ybits) | (u64)(u32)(p.y - y0);
        const u32 wbin = (u32)(key >> wshift);
        atomicMax(&S.wkey[(c > 0 ? 0 : BW_BINS) + wbin], ((u64)quant << 32) | (u64)(i + 1u));
      }
      }
    }
    __syncthreads();
    // Every bin's exclusive prefix maximum, per region (thread t owns bins
    // [t BW_PER, (t + 1) BW_PER)), and its witness direction.
    {
      constexpr int BW_PER = (BW_BINS + BLOCK - 1) / BLOCK;
      for (int r = 0; r < 2; ++r) {
        u64 v[BW_PER];
        u64 tot = 0;
        #pragma unroll
        for (int q = 0; q < BW_PER; ++q) {
          const int bq = threadIdx.x * BW_PER + q;
          v[q] = bq < BW_BINS ? S.wkey[r * BW_BINS + bq] : 0ull;
          tot = v[q] > tot ? v[q] : tot;
        }
        u64 inc = tot;
        #pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const u64 t = __shfl_up_sync(0xFFFFFFFFu, inc, o);
          if (lane >= o && t > inc) inc = t;
        }
        u64 ex = __shfl_up_sync(0xFFFFFFFFu, inc, 1);
        if (lane == 0) ex = 0;
        if (lane == 31) S.wmax[wid] = inc;
        __syncthreads();
        for (int w = 0; w < wid; ++w) ex = S.wmax[w] > ex ? S.wmax[w] : ex;
        #pragma unroll
        for (int q = 0; q < BW_PER; ++q) {
          const int bq = threadIdx.x * BW_PER + q;
          const u32 wi = (u32)ex;                // sample index + 1, 0: none (P_0 itself)
          if (bq < BW_BINS) {
            int2 w = make_int2(d0x, d0y);
            if (wi) { const int2 p = __ldcg(&smp[wi - 1u]); w = make_int2(p.x - bxp, p.y - byp); }
            S.wtab[2 * bq + r] = w;
          }
          ex = v[q] > ex ? v[q] : ex;
        }
        __syncthreads();
      }
    }
    if (MODE == 1) {
      // The record k_seg_filter and mode 2 read: plan, edges, witness table.
      SegRec& R = a.rec[S.hq];
      if (threadIdx.x == 0) R.plan = S.plan;
      for (int q = threadIdx.x; q < kMaxCorners; q += BLOCK) R.edge[q] = S.edge[q];
      for (int q = threadIdx.x; q < 2 * BW_BINS; q += BLOCK) R.wtab[q] = S.wtab[q];
      __syncthreads();
      continue;
    }
    }   // modes 0, 1

    // ---- 2. witness test, filter polygon and compaction (+ digit
    // histograms).  Warp w takes the round's points [base + w WSPAN, base +
    // (w + 1) WSPAN), so the survivors come out in input order; the next
    // round's points are loaded before this round's scan.
    constexpr u32 WSPAN = 32u * BT_FITEMS;
    u32* bcnt = &S.hist[0][0];          // survivors per witness bin (zeroed with the histograms)
    u32* bcur = &S.hist[2][0];
    u32 run = 0;
    if (MODE == 2) {
      // The survivors k_seg_filter left at the start of every tile run
      // (runs in tile order, each run's survivors in no particular order),
      // gathered and counted per witness bin: the instance's survivor i (in
      // run order) lies in the last tile whose run start is at most i.  An
      // instance has at most 128 tiles (batch_max_instance() points), fewer
      // than BLOCK.
      const int tf = a.tfirst[S.hq], nt = a.tfirst[S.hq + 1] - tf;
      const u32 c = (int)threadIdx.x < nt ? a.tcnt[tf + threadIdx.x] : 0u;
      u32 inc = c;
      #pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const u32 t = __shfl_up_sync(0xFFFFFFFFu, inc, o);
        if (lane >= o) inc += t;
      }
      if (lane == 31) S.red[wid] = inc;
      __syncthreads();
      u32 ex = inc - c, tot = 0;
      for (int w = 0; w < W; ++w) { if (w < wid) ex += S.red[w]; tot += S.red[w]; }
      if ((int)threadIdx.x < nt) S.chunk_cnt[threadIdx.x] = (int)ex;
      __syncthreads();
      for (u32 i0 = threadIdx.x; i0 < tot; i0 += 4 * BLOCK) {   // four loads in flight per thread
        u64 k[4];
        u32 v[4];
        #pragma unroll
        for (int r = 0; r < 4; ++r) {
          const u32 i = i0 + r * BLOCK;
          k[r] = 0ull;
          v[r] = 0u;
          if (i < tot) {
            int lo = 0, hi = nt - 1;
            while (lo < hi) {
              const int mid = (lo + hi + 1) >> 1;
              if ((u32)S.chunk_cnt[mid] <= i) lo = mid; else hi = mid - 1;
            }
            const long long src = sl + (long long)lo * SEG_TILE + (i - (u32)S.chunk_cnt[lo]);
            k[r] = __ldcg(&a.kb[src]);
            v[r] = __ldcg(&a.ib[src]);
          }
        }
        #pragma unroll
        for (int r = 0; r < 4; ++r) {
          const u32 i = i0 + r * BLOCK;
          if (i < tot) {
            if (i < n) {
              a.ka[sl + i] = k[r];
              a.ia[sl + i] = v[r];
            }
            atomicAdd(&bcnt[(u32)(k[r] >> wshift)], 1u);
          }
        }
      }
      run = tot < n ? tot : n;
      __syncthreads();
    } else {
    int2 cur[BT_FITEMS];
    #pragma unroll
    for (int r = 0; r < BT_FITEMS; ++r) {
      const u32 j = wid * WSPAN + r * 32 + lane;
      cur[r] = j < n ? P[j] : make_int2(0, 0);
    }
    u32 parity = 0;
    for (u32 base = 0; base < n; base += FCH, parity ^= 1u) {
      const u32 j0 = base + wid * WSPAN + lane;
      u32 kmask = 0;
      #pragma unroll
      for (int r = 0; r < BT_FITEMS; ++r) {        // the witness test of the point's bin and region
        if (j0 + r * 32 < n) {
          const int dx = cur[r].x - bxp, dy = cur[r].y - byp;
          const long long c = cross2(d0x, d0y, dx, dy);
          const u32 xr = (u32)(cur[r].x - x0);
          const u32 wb = wx_only ? xr >> wsx : (xr << wsx) | ((u32)(cur[r].y - y0) >> wshift);
          const int2 w = S.wtab[2 * wb + (c < 0 ? 1u : 0u)];
          const long long t = cross2(w.x, w.y, dx, dy);
          if (c == 0 || (c > 0 ? t > 0 : t < 0)) kmask |= 1u << r;
        }
      }
      // The witness survivors staged in the warp's slice, in input order
      // (a few per round); the filter polygon on them, one per lane; the
      // warps' kept counts scanned across the block; the kept ones written
      // in input order.
      u32 wc = 0;
      #pragma unroll
      for (int r = 0; r < BT_FITEMS; ++r) {
        const u32 bal = __ballot_sync(0xFFFFFFFFu, (kmask >> r) & 1u);
        if ((kmask >> r) & 1u) {
          const u32 q = wc + __popc(bal & lt_mask);
          S.st.sxy[wid][q] = cur[r];
          S.st.sidx[wid][q] = j0 + r * 32;
        }
        wc += __popc(bal);
      }
      __syncwarp();
      u32 kb[BT_FITEMS], kc = 0;
      #pragma unroll
      for (int c = 0; c < BT_FITEMS; ++c) {
        const u32 q = c * 32 + lane;
        bool keep = false;
        if (q < wc) {
          const int2 p = S.st.sxy[wid][q];
          keep = !in_polygon(S.edge, ncorner, p.x, p.y);
        }
        kb[c] = (u32)c * 32 < wc ? __ballot_sync(0xFFFFFFFFu, keep) : 0u;
        kc += __popc(kb[c]);
      }
      u32* red = S.red + parity * (W + 1);
      if (lane == 0) red[wid] = kc;
      int2 nxt[BT_FITEMS];
      #pragma unroll
      for (int r = 0; r < BT_FITEMS; ++r) {
        const u32 j = j0 + FCH + r * 32;
        nxt[r] = j < n ? P[j] : make_int2(0, 0);
      }
      __syncthreads();
      if (wid == 0) {
        const u32 v = lane < W ? red[lane] : 0u;
        u32 inc = v;
        #pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const u32 t = __shfl_up_sync(0xFFFFFFFFu, inc, o);
          if (lane >= o) inc += t;
        }
        if (lane < W) red[lane] = inc - v;
        if (lane == W - 1) red[W] = inc;
      }
      __syncthreads();
      u32 pos = run + red[wid];
      #pragma unroll
      for (int c = 0; c < BT_FITEMS; ++c) {
        if ((kb[c] >> lane) & 1u) {
          const u32 q = c * 32 + lane;
          const int2 p = S.st.sxy[wid][q];
          const u32 o = pos + __popc(kb[c] & lt_mask);
          const u64 key = ((u64)(u32)(p.x - x0) << ybits) | (u64)(u32)(p.y - y0);
          if (o < n) {
            a.ka[sl + o] = key;
            a.ia[sl + o] = S.st.sidx[wid][q];
          }
          atomicAdd(&bcnt[(u32)(key >> wshift)], 1u);
        }
        pos += __popc(kb[c]);
      }
      __syncwarp();
      run += red[W];
      #pragma unroll
      for (int r = 0; r < BT_FITEMS; ++r) cur[r] = nxt[r];
    }
    }   // mode 0
    __syncthreads();
    const u32 s = run;

    // ---- 3. sort (step 4) by (key, index), the order of a stable sort of
    // the keys in input order, into the second key / index buffers.  Up to
    // SCAP survivors: moved into shared memory by witness bin (the key's top
    // bits, so the bins are in key order), then every bin sorted
    // (sort_bins_out: by rank, or by the block's bitonic network).  More,
    // with no bin above SCAP: moved into bin order in the scratch region,
    // then groups of consecutive bins of at most SCAP survivors each sorted
    // the same way through shared memory.  Otherwise (thousands of equal
    // keys): a stable LSD radix sort through the scratch region (digit
    // histograms first).
    const u64* rs_k;
    const u32* rs_i;
    {
        constexpr int PER = BW_BINS / BLOCK > 0 ? BW_BINS / BLOCK : 1;
        u32 v[PER], tot = 0;
        #pragma unroll
        for (int q = 0; q < PER; ++q) {
          const int b = threadIdx.x * PER + q;
          v[q] = b < BW_BINS ? bcnt[b] : 0u;
          tot += v[q];
        }
        u32 inc = tot;
        #pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const u32 t = __shfl_up_sync(0xFFFFFFFFu, inc, o);
          if (lane >= o) inc += t;
        }
        if (lane == 31) S.red[wid] = inc;
        if (threadIdx.x == 0) S.nbig = 0;
        __syncthreads();
        u32 ex = inc - tot;
        for (int w = 0; w < wid; ++w) ex += S.red[w];
        #pragma unroll
        for (int q = 0; q < PER; ++q) {
          const int b = threadIdx.x * PER + q;
          if (b < BW_BINS) bcur[b] = ex;
          ex += v[q];
        }
        if (threadIdx.x == 0) S.ngrp = 0;
        __syncthreads();
    }
    if (s > (u32)Smem<BLOCK>::SCAP && threadIdx.x == 0) {
      // Groups of consecutive bins, greedily up to SCAP survivors each
      // (their first bins in S.big); none when a bin alone exceeds SCAP.
      u32 ng = 0, acc = 0;
      bool ok = true;
      for (u32 b = 0; b < (u32)BW_BINS && ok; ++b) {
        const u32 c = bcnt[b];
        ok = c <= (u32)Smem<BLOCK>::SCAP;
        if (ng == 0 || acc + c > (u32)Smem<BLOCK>::SCAP) { S.big[ng++] = (unsigned short)b; acc = 0; }
        acc += c;
      }
      S.ngrp = ok ? ng : 0u;
    }
    __syncthreads();
    if (s <= (u32)Smem<BLOCK>::SCAP) {
      for (u32 i = threadIdx.x; i < s; i += BLOCK) {
        const u64 k = __ldcg(&a.ka[sl + i]);
        const u32 q = atomicAdd(&bcur[(u32)(k >> wshift)], 1u);   // bcur[b]: the bin's end after
        S.bk[q] = k;
        S.bi[q] = __ldcg(&a.ia[sl + i]);
      }
      __syncthreads();
      sort_bins_out<BLOCK>(S, bcnt, bcur, 0u, (u32)BW_BINS, 0u, s, wshift, a.kb + sl, a.ib + sl);
      rs_k = a.kb + sl;
      rs_i = a.ib + sl;
    } else if (S.ngrp > 0) {
      for (u32 i0 = threadIdx.x; i0 < s; i0 += 4 * BLOCK) {   // four loads in flight per thread
        u64 k[4];
        u32 v[4];
        #pragma unroll
        for (int r = 0; r < 4; ++r) {
          const u32 i = i0 + r * BLOCK;
          k[r] = i < s ? __ldcg(&a.ka[sl + i]) : 0ull;
          v[r] = i < s ? __ldcg(&a.ia[sl + i]) : 0u;
        }
        #pragma unroll
        for (int r = 0; r < 4; ++r) {
          if (i0 + r * BLOCK < s) {
            const u32 q = atomicAdd(&bcur[(u32)(k[r] >> wshift)], 1u);   // bcur[b]: the bin's end after
            a.kb[sl + q] = k[r];
            a.ib[sl + q] = v[r];
          }
        }
      }
      __syncthreads();
      const u32 ng = S.ngrp;
      for (u32 g = 0; g < ng; ++g) {
        const u32 g0 = S.big[g], g1 = g + 1 < ng ? (u32)S.big[g + 1] : (u32)BW_BINS;
        const u32 p0 = bcur[g0] - bcnt[g0], p1 = bcur[g1 - 1];
        for (u32 i = threadIdx.x; i < p1 - p0; i += BLOCK) {
          S.bk[i] = __ldcg(&a.kb[sl + p0 + i]);
          S.bi[i] = __ldcg(&a.ib[sl + p0 + i]);
        }
        __syncthreads();
        sort_bins_out<BLOCK>(S, bcnt, bcur, g0, g1, p0, p1 - p0, wshift, a.kb + sl, a.ib + sl);
      }
      rs_k = a.kb + sl;
      rs_i = a.ib + sl;
    } else {
    for (int q = threadIdx.x; q < kMaxPasses * kRadix; q += BLOCK) (&S.hist[0][0])[q] = 0u;
    __syncthreads();
    for (u32 i = threadIdx.x; i < s; i += BLOCK) {
      const u64 key = __ldcg(&a.ka[sl + i]);
      for (u32 p = 0; p < npasses; ++p)
        atomicAdd(&S.hist[p][(u32)(key >> (p * kRadixBits)) & (kRadix - 1)], 1u);
    }
    __syncthreads();
    u64* src_k = a.ka + sl; u32* src_i = a.ia + sl;
    u64* dst_k = a.kb + sl; u32* dst_i = a.ib + sl;
    // Mode 2's survivors are in no particular order within a tile run:
    // passes over the index digits come first, so that the stable passes
    // over the key leave equal keys in index order.
    const u32 ipasses = MODE == 2 ? (bitlen32(n - 1u) + kRadixBits - 1) / kRadixBits : 0u;
    for (u32 pass = 0; pass < ipasses + npasses; ++pass) {
      const bool by_idx = MODE == 2 && pass < ipasses;
      const u32 shift = (by_idx ? pass : pass - ipasses) * kRadixBits;
      if (by_idx) {   // the index digits' histogram, in the first warp slot of the tile counters
        for (int q = threadIdx.x; q < kRadix; q += BLOCK) S.wpos[0][q] = 0u;
        __syncthreads();
        for (u32 i = threadIdx.x; i < s; i += BLOCK) atomicAdd(&S.wpos[0][(src_i[i] >> shift) & (kRadix - 1)], 1u);
        __syncthreads();
      }
      // Exclusive start of every digit inside the instance's range.
      u32 hv = 0, hinc = 0;
      if (threadIdx.x < kRadix) {
        hv = by_idx ? S.wpos[0][threadIdx.x] : S.hist[pass - ipasses][threadIdx.x];
        hinc = hv;
        #pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const u32 t = __shfl_up_sync(0xFFFFFFFFu, hinc, o);
          if (lane >= o) hinc += t;
        }
        if (lane == 31) S.red[wid] = hinc;
      }
      __syncthreads();
      if (threadIdx.x < kRadix) {
        u32 o2 = 0;
        for (int w = 0; w < wid; ++w) o2 += S.red[w];
        S.cur[threadIdx.x] = o2 + hinc - hv;
      }
      __syncthreads();
      for (u32 tb = 0; tb < s; tb += TILE) {
        for (int q = threadIdx.x; q < W * kRadix; q += BLOCK) (&S.wpos[0][0])[q] = 0u;
        __syncthreads();
        u64 key[BT_ITEMS];
        u32 idv[BT_ITEMS];
        const u32 wb = tb + wid * 32 * BT_ITEMS;
        #pragma unroll
        for (int it = 0; it < BT_ITEMS; ++it) {
          const u32 p = wb + it * 32 + lane;
          key[it] = p < s ? src_k[p] : 0ull;
          idv[it] = p < s ? src_i[p] : 0u;
          const u32 dg = by_idx ? (idv[it] >> shift) & (kRadix - 1) : (u32)(key[it] >> shift) & (kRadix - 1);
          if (p < s) atomicAdd(&S.wpos[wid][dg], 1u);
        }
        __syncthreads();
        if (threadIdx.x < kRadix) {
          const int d = threadIdx.x;
          u32 r2 = S.cur[d];
          #pragma unroll
          for (int w = 0; w < W; ++w) { const u32 c = S.wpos[w][d]; S.wpos[w][d] = r2; r2 += c; }
          S.cur[d] = r2;
        }
        __syncthreads();
        #pragma unroll
        for (int it = 0; it < BT_ITEMS; ++it) {
          const u32 p = wb + it * 32 + lane;
          const bool valid = p < s;
          const u32 dg = by_idx ? (idv[it] >> shift) & (kRadix - 1) : (u32)(key[it] >> shift) & (kRadix - 1);
          const u32 peers = warp_digit_peers(dg) & __ballot_sync(0xFFFFFFFFu, valid);
          const int leader = 31 - __clz(peers);
          u32 pos = 0;
          if (valid && lane == leader) pos = atomicAdd(&S.wpos[wid][dg], (u32)__popc(peers));
          pos = __shfl_sync(0xFFFFFFFFu, pos, valid ? leader : lane) + __popc(peers & lt_mask);
          if (valid && pos < s) { dst_k[pos] = key[it]; dst_i[pos] = idv[it]; }
        }
        __syncthreads();
      }
      u64* tk = src_k; src_k = dst_k; dst_k = tk;
      u32* ti = src_i; src_i = dst_i; dst_i = ti;
    }
    rs_k = src_k;
    rs_i = src_i;
    }
    __syncthreads();

    // ---- 4. region split + second round (running prefix of directions)
    int2* LX = a.lxy + sl; int* LI = a.lidx + sl;
    int2* UX = a.uxy + sl; int* UI = a.uidx + sl;
    if (ax == bxp && ay == byp) {   // every point equal: one vertex
      if (threadIdx.x == 0) { a.out_tmp[sl] = ext0; a.hcount[inst] = 1; }
      __syncthreads();
      continue;
    }
    const u64 ymask = ybits ? ((~0ull) >> (64 - ybits)) : 0ull;
    Dir2b R = {d0x, d0y, d0x, d0y};
    u32 rl = 0, ru = 0;
    for (u32 cb = 0; cb < s; cb += FCH) {
      int px[BT_FITEMS], py[BT_FITEMS], pi[BT_FITEMS];
      signed char side[BT_FITEMS];
      const u32 first = cb + threadIdx.x * BT_FITEMS;
      Dir2b ag = {d0x, d0y, d0x, d0y};
      #pragma unroll
      for (int i = 0; i < BT_FITEMS; ++i) {
        const u32 p = first + i;
        side[i] = 0; px[i] = 0; py[i] = 0; pi[i] = 0;
        if (p < s) {
          const u64 k = rs_k[p];
          px[i] = x0 + (int)(u32)(k >> ybits);
          py[i] = y0 + (int)(u32)(k & ymask);
          pi[i] = (int)rs_i[p];
          const long long o = cross2(ux, uy, px[i] - ax, py[i] - ay);
          side[i] = o < 0 ? -1 : (o > 0 ? 1 : 0);
          const int vx = px[i] - bxp, vy = py[i] - byp;
          if (side[i] < 0 && cross2(ag.lx, ag.ly, vx, vy) > 0) { ag.lx = vx; ag.ly = vy; }
          if (side[i] > 0 && cross2(ag.ux, ag.uy, vx, vy) < 0) { ag.ux = vx; ag.uy = vy; }
        }
      }
      Dir2b inc = ag;
      #pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        Dir2b t = dshfl_up(inc, o);
        if (lane >= o) { dcombine(t, inc); inc = t; }
      }
      Dir2b lex = dshfl_up(inc, 1);
      if (lane == 31) S.wdir[wid] = inc;
      __syncthreads();
      Dir2b runv = R;
      for (int w = 0; w < wid; ++w) dcombine(runv, S.wdir[w]);
      if (lane > 0) dcombine(runv, lex);
      unsigned kl = 0, ku = 0;
      #pragma unroll
      for (int i = 0; i < BT_FITEMS; ++i) {
        const int vx = px[i] - bxp, vy = py[i] - byp;
        if (side[i] < 0) {
          if (cross2(runv.lx, runv.ly, vx, vy) > 0) { kl |= 1u << i; runv.lx = vx; runv.ly = vy; }
        } else if (side[i] > 0) {
          if (cross2(runv.ux, runv.uy, vx, vy) < 0) { ku |= 1u << i; runv.ux = vx; runv.uy = vy; }
        }
      }
      const u32 cl = __popc(kl), cu = __popc(ku);
      u32 il = cl, iu = cu;
      #pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const u32 t0 = __shfl_up_sync(0xFFFFFFFFu, il, o), t1 = __shfl_up_sync(0xFFFFFFFFu, iu, o);
        if (lane >= o) { il += t0; iu += t1; }
      }
      if (lane == 31) { S.wcnt[wid][0] = il; S.wcnt[wid][1] = iu; }
      __syncthreads();
      u32 wl = 0, wu = 0, tl = 0, tu = 0;
      Dir2b cagg = R;
      for (int w = 0; w < W; ++w) {
        if (w < wid) { wl += S.wcnt[w][0]; wu += S.wcnt[w][1]; }
        tl += S.wcnt[w][0]; tu += S.wcnt[w][1];
        dcombine(cagg, S.wdir[w]);
      }
      u32 pl0 = 1 + rl + wl + il - cl, pu0 = 1 + ru + wu + iu - cu;
      #pragma unroll
      for (int i = 0; i < BT_FITEMS; ++i) {
        if (kl & (1u << i)) { if (pl0 < s + 1) { LX[pl0] = make_int2(px[i], py[i]); LI[pl0] = pi[i]; } ++pl0; }
        else if (ku & (1u << i)) { if (pu0 < s + 1) { UX[pu0] = make_int2(px[i], py[i]); UI[pu0] = pi[i]; } ++pu0; }
      }
      R = cagg;
      rl += tl; ru += tu;
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      LX[0] = make_int2(ax, ay); LI[0] = ext0;
      UX[0] = make_int2(ax, ay); UI[0] = ext0;
      LX[rl + 1] = make_int2(bxp, byp); LI[rl + 1] = ext1;
      UX[ru + 1] = make_int2(bxp, byp); UI[ru + 1] = ext1;
    }
    __syncthreads();

    // ---- 5. chains (scratch: the sort buffers, free now), 6. staged output
    int2* g0 = reinterpret_cast<int2*>(a.ka + sl);
    int2* g1 = reinterpret_cast<int2*>(a.kb + sl);
    int* g0i = reinterpret_cast<int*>(a.ia + sl);
    int* g1i = reinterpret_cast<int*>(a.ib + sl);
    int* out = a.out_tmp + sl;
    int where = 0;
    const int hl = build_chain<BLOCK>(S, LX, LI, (int)rl + 2, 1, g0, g0i, g1, g1i, &where);
    for (int i = threadIdx.x; i < hl; i += BLOCK)
      out[i] = where == 0 ? S.si[i] : (where == 1 ? __ldcg(&g0i[i]) : __ldcg(&g1i[i]));
    __syncthreads();
    const int hu = build_chain<BLOCK>(S, UX, UI, (int)ru + 2, -1, g0, g0i, g1, g1i, &where);
    for (int k = threadIdx.x; k < hu - 2; k += BLOCK) {
      const int q = hu - 2 - k;
      out[hl + k] = where == 0 ? S.si[q] : (where == 1 ? __ldcg(&g0i[q]) : __ldcg(&g1i[q]));
    }
    if (threadIdx.x == 0) a.hcount[inst] = (u32)(hl + hu - 2);
    __syncthreads();
  }
}

// Output: exclusive scan of the hull sizes, then every hull copied to its
// offset (single block for the scan, all blocks for the copy).
__global__ void k_batch_scan(const u32* __restrict__ hcount, int B, long long* out_off, long long cap,
                             u32* error) {
  __shared__ long long s_w[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int per = (B + blockDim.x - 1) / blockDim.x;
  const int lo = min(B, (int)threadIdx.x * per), hi = min(B, lo + per);
  long long sum = 0;
  for (int i = lo; i < hi; ++i) sum += hcount[i];
  long long inc = sum;
  #pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const long long t = __shfl_up_sync(0xFFFFFFFFu, inc, o);
    if (lane >= o) inc += t;
  }
  if (lane == 31) s_w[wid] = inc;
  __syncthreads();
  long long off = 0;
  for (int w = 0; w < wid; ++w) off += s_w[w];
  long long r = off + inc - sum;
  for (int i = lo; i < hi; ++i) { out_off[i] = r; r += hcount[i]; }
  if (threadIdx.x == blockDim.x - 1) {
    out_off[B] = off + inc;
    if (off + inc > cap) atomicOr(error, ERR_CAPACITY);
  }
}

__global__ void k_batch_copy(const u32* __restrict__ hcount, const long long* __restrict__ slot0,
                             const int* __restrict__ out_tmp, const long long* __restrict__ out_off,
                             int B, int* out, long long cap) {
  if (out_off[B] > cap) return;
  for (int i = blockIdx.x; i < B; i += gridDim.x) {
    const u32 h = hcount[i];
    const long long o = out_off[i], s0 = slot0[i];
    for (u32 j = threadIdx.x; j < h; j += blockDim.x) out[o + j] = out_tmp[s0 + j];
  }
}

// ---------------------------------------------------------------- segmented
// The two streaming passes of the largest instances, flat over all their
// tiles: block b takes the consecutive tiles [b T / G, (b + 1) T / G), split
// into runs of one instance each, so every block streams an equal share of
// the points whatever the instances' sizes.

// The instance (position in `order`) of tile t: the last h with tfirst[h] <= t.
__device__ __forceinline__ int seg_of_tile(const int* __restrict__ tfirst, int nh, int t) {
  int lo = 0, hi = nh - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (tfirst[mid] <= t) lo = mid; else hi = mid - 1;
  }
  return lo;
}

constexpr int SEG_BLOCK = 512;

// Pass 1: the extremes of every tile run (step 1: as the whole-pipeline
// kernel, with the skip box of the run's first round), written to the run's
// first tile (the run's other tiles get none), and every BW_STRIDE-th point
// of the instance copied to its sample.
__global__ void __launch_bounds__(SEG_BLOCK)
k_seg_ext(BatchArgs a, int ntiles) {
  constexpr int W = SEG_BLOCK / 32;
  constexpr u32 FCH = SEG_BLOCK * BT_FITEMS;
  __shared__ int s_box[4];
  __shared__ u64 s_rk[W][4];
  __shared__ u32 s_ri[W][4];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int t1 = (int)(((long long)(blockIdx.x + 1) * ntiles) / gridDim.x);
  int t = (int)(((long long)blockIdx.x * ntiles) / gridDim.x);
  while (t < t1) {
    const int h = seg_of_tile(a.tfirst, a.nb, t);
    const int tf = a.tfirst[h], te = min(t1, a.tfirst[h + 1]);
    const int inst = a.order[h];
    const long long off = a.offsets[inst];
    const u32 n = (u32)(a.offsets[inst + 1] - off);
    const int2* P = reinterpret_cast<const int2*>(a.xy) + off;
    int2* smp = reinterpret_cast<int2*>(a.kb + a.slot0[inst]);
    const u32 lo = (u32)(t - tf) * SEG_TILE;
    const u32 hi = min(n, (u32)(te - tf) * SEG_TILE);
    if (threadIdx.x == 0) {
      s_box[0] = 0x7FFFFFFF; s_box[1] = (int)0x80000000; s_box[2] = 0x7FFFFFFF; s_box[3] = (int)0x80000000;
    }
    __syncthreads();
    int2 p[BT_FITEMS];
    {
      int x0 = 0x7FFFFFFF, x1 = (int)0x80000000, y0 = 0x7FFFFFFF, y1 = (int)0x80000000;
      #pragma unroll
      for (int r = 0; r < BT_FITEMS; ++r) {
        const u32 j = lo + r * SEG_BLOCK + threadIdx.x;
        p[r] = j < hi ? P[j] : make_int2(0, 0);
        if (j < hi) {
          x0 = min(x0, p[r].x); x1 = max(x1, p[r].x); y0 = min(y0, p[r].y); y1 = max(y1, p[r].y);
        }
      }
      #pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        x0 = min(x0, __shfl_xor_sync(0xFFFFFFFFu, x0, o)); x1 = max(x1, __shfl_xor_sync(0xFFFFFFFFu, x1, o));
        y0 = min(y0, __shfl_xor_sync(0xFFFFFFFFu, y0, o)); y1 = max(y1, __shfl_xor_sync(0xFFFFFFFFu, y1, o));
      }
      if (lane == 0 && x0 <= x1) {
        atomicMin(&s_box[0], x0); atomicMax(&s_box[1], x1); atomicMin(&s_box[2], y0); atomicMax(&s_box[3], y1);
      }
    }
    __syncthreads();
    const int kx0 = s_box[0], kx1 = s_box[1], ky0 = s_box[2], ky1 = s_box[3];
    BestX b;
    bx_init(b);
    for (u32 base = lo; base < hi; base += FCH) {
      int2 q[BT_FITEMS];
      #pragma unroll
      for (int r = 0; r < BT_FITEMS; ++r) {
        const u32 j = base + FCH + r * SEG_BLOCK + threadIdx.x;
        q[r] = j < hi ? P[j] : make_int2(0, 0);
      }
      #pragma unroll
      for (int r = 0; r < BT_FITEMS; ++r) {
        const u32 j = base + r * SEG_BLOCK + threadIdx.x;
        if (j < hi) {
          if (!(p[r].x > kx0 && p[r].x < kx1 && p[r].y > ky0 && p[r].y < ky1)) bx_point(b, p[r].x, p[r].y, j);
          if (j % BW_STRIDE == 0) smp[j / BW_STRIDE] = p[r];
        }
      }
      #pragma unroll
      for (int r = 0; r < BT_FITEMS; ++r) p[r] = q[r];
    }
    bx_warp(b);
    if (lane == 0)
      for (int q = 0; q < 4; ++q) { s_rk[wid][q] = b.k[q]; s_ri[wid][q] = b.i[q]; }
    __syncthreads();
    if (threadIdx.x == 0) {
      bx_init(b);
      for (int w = 0; w < W; ++w) bx_merge(b, s_rk[w], s_ri[w]);
      for (int j = 0; j < 4; ++j) { a.text[t].k[j] = b.k[j]; a.text[t].i[j] = b.i[j]; }
    }
    for (int u = t + 1 + (int)threadIdx.x; u < te; u += SEG_BLOCK)
      for (int j = 0; j < 4; ++j) { a.text[u].k[j] = ~0ull; a.text[u].i[j] = 0xFFFFFFFFu; }
    __syncthreads();
    t = te;
  }
}

// Pass 2: the witness test of the point's bin and region, then the filter
// polygon on the witness survivors (step 2 of the whole-pipeline kernel,
// from the instance's record), compacted to the start of the run's range of
// the instance's second key / index buffers: every warp reserves its
// round's survivors with one shared-memory atomic, so no block barrier
// stands in the stream and the survivors of a run are in no particular
// order (the sort orders (key, index) pairs; its radix fallback sorts by
// index first).  The count goes to the run's first tile (0 for its other
// tiles).
__global__ void __launch_bounds__(SEG_BLOCK)
k_seg_filter(BatchArgs a, int ntiles) {
  constexpr u32 FCH = SEG_BLOCK * BT_FITEMS;
  constexpr u32 WSPAN = 32u * BT_FITEMS;
  constexpr int W = SEG_BLOCK / 32;
  __shared__ IPlan s_plan;
  __shared__ int4 s_edge[kMaxCorners];
  __shared__ int2 s_wtab[2 * BW_BINS];
  __shared__ int2 s_sxy[W][WSPAN];   // per warp: the round's witness survivors, staged
  __shared__ u32 s_sidx[W][WSPAN];
  __shared__ u32 s_cnt;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const u32 lt_mask = (1u << lane) - 1u;
  const int t1 = (int)(((long long)(blockIdx.x + 1) * ntiles) / gridDim.x);
  int t = (int)(((long long)blockIdx.x * ntiles) / gridDim.x);
  while (t < t1) {
    const int h = seg_of_tile(a.tfirst, a.nb, t);
    const int tf = a.tfirst[h], te = min(t1, a.tfirst[h + 1]);
    const int inst = a.order[h];
    const long long off = a.offsets[inst];
    const u32 n = (u32)(a.offsets[inst + 1] - off);
    const long long sl = a.slot0[inst];
    const int2* P = reinterpret_cast<const int2*>(a.xy) + off;
    const SegRec& R = a.rec[h];
    if (threadIdx.x == 0) { s_plan = R.plan; s_cnt = 0; }
    for (int q = threadIdx.x; q < kMaxCorners; q += SEG_BLOCK) s_edge[q] = R.edge[q];
    for (int q = threadIdx.x; q < 2 * BW_BINS; q += SEG_BLOCK) s_wtab[q] = R.wtab[q];
    __syncthreads();
    const u32 lo = (u32)(t - tf) * SEG_TILE;
    const u32 hi = min(n, (u32)(te - tf) * SEG_TILE);
    if (!s_plan.bad) {
      const int bxp = s_plan.ext_x[1], byp = s_plan.ext_y[1];
      const int d0x = s_plan.ext_x[0] - bxp, d0y = s_plan.ext_y[0] - byp;
      const int x0 = s_plan.x0, y0 = s_plan.y0, ncorner = s_plan.ncorner;
      const u32 ybits = s_plan.ybits, kbits = s_plan.kbits;
      const u32 wshift = kbits > (u32)BW_BITS ? kbits - (u32)BW_BITS : 0u;
      const bool wx_only = wshift >= ybits;
      const u32 wsx = wx_only ? wshift - ybits : ybits - wshift;
      int2 cur[BT_FITEMS];
      #pragma unroll
      for (int r = 0; r < BT_FITEMS; ++r) {
        const u32 j = lo + wid * WSPAN + r * 32 + lane;
        cur[r] = j < hi ? P[j] : make_int2(0, 0);
      }
      for (u32 base = lo; base < hi; base += FCH) {
        const u32 j0 = base + wid * WSPAN + lane;
        u32 kmask = 0;
        #pragma unroll
        for (int r = 0; r < BT_FITEMS; ++r) {
          if (j0 + r * 32 < hi) {
            const int dx = cur[r].x - bxp, dy = cur[r].y - byp;
            const long long c = cross2(d0x, d0y, dx, dy);
            const u32 xr = (u32)(cur[r].x - x0);
            const u32 wb = wx_only ? xr >> wsx : (xr << wsx) | ((u32)(cur[r].y - y0) >> wshift);
            const int2 w = s_wtab[2 * wb + (c < 0 ? 1u : 0u)];
            const long long tt = cross2(w.x, w.y, dx, dy);
            if (c == 0 || (c > 0 ? tt > 0 : tt < 0)) kmask |= 1u << r;
          }
        }
        // The witness survivors staged in the warp's slice (a few per
        // round), then the filter polygon on them, one per lane, and the
        // kept ones reserved with one shared-memory atomic per 32.
        u32 wc = 0;
        #pragma unroll
        for (int r = 0; r < BT_FITEMS; ++r) {
          const u32 bal = __ballot_sync(0xFFFFFFFFu, (kmask >> r) & 1u);
          if ((kmask >> r) & 1u) {
            const u32 q = wc + __popc(bal & lt_mask);
            s_sxy[wid][q] = cur[r];
            s_sidx[wid][q] = j0 + r * 32;
          }
          wc += __popc(bal);
        }
        int2 nxt[BT_FITEMS];
        #pragma unroll
        for (int r = 0; r < BT_FITEMS; ++r) {
          const u32 j = j0 + FCH + r * 32;
          nxt[r] = j < hi ? P[j] : make_int2(0, 0);
        }
        __syncwarp();
        for (u32 q0 = 0; q0 < wc; q0 += 32) {
          const u32 q = q0 + lane;
          int2 p = make_int2(0, 0);
          bool keep = false;
          if (q < wc) {
            p = s_sxy[wid][q];
            keep = !in_polygon(s_edge, ncorner, p.x, p.y);
          }
          const u32 kb = __ballot_sync(0xFFFFFFFFu, keep);
          u32 pos = 0;
          if (lane == 0 && kb) pos = atomicAdd(&s_cnt, (u32)__popc(kb));
          pos = __shfl_sync(0xFFFFFFFFu, pos, 0) + __popc(kb & lt_mask);
          if (keep && lo + pos < n) {
            a.kb[sl + lo + pos] = ((u64)(u32)(p.x - x0) << ybits) | (u64)(u32)(p.y - y0);
            a.ib[sl + lo + pos] = s_sidx[wid][q];
          }
        }
        __syncwarp();
        #pragma unroll
        for (int r = 0; r < BT_FITEMS; ++r) cur[r] = nxt[r];
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) a.tcnt[t] = s_cnt;
    for (int u = t + 1 + (int)threadIdx.x; u < te; u += SEG_BLOCK) a.tcnt[u] = 0;
    __syncthreads();
    t = te;
  }
}

BatchArgs batch_args(const BatchLaunch& L) {
  BatchArgs a;
  a.xy = L.xy; a.offsets = L.offsets; a.order = L.order; a.nb = L.nb; a.queue = L.queue;
  a.slot0 = L.slot0; a.ka = L.ka; a.kb = L.kb; a.ia = L.ia; a.ib = L.ib;
  a.lxy = L.lxy; a.lidx = L.lidx; a.uxy = L.uxy; a.uidx = L.uidx;
  a.out_tmp = L.out_tmp; a.hcount = L.hcount; a.error = L.error;
  a.w16 = reinterpret_cast<const __half*>(L.w16);
  a.mode = L.mode; a.tfirst = L.tfirst;
  a.text = reinterpret_cast<SegTileExt*>(L.text);
  a.tcnt = L.tcnt;
  a.rec = reinterpret_cast<SegRec*>(L.rec);
  return a;
}

}  // namespace

int seg_tile() { return (int)SEG_TILE; }
size_t seg_rec_bytes() { return sizeof(SegRec); }
size_t seg_text_bytes() { return sizeof(SegTileExt); }

cudaError_t seg_configure(int* occ_ext, int* occ_filter) {
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ_ext, k_seg_ext, SEG_BLOCK, 0);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ_filter, k_seg_filter, SEG_BLOCK, 0);
}

cudaError_t launch_seg_ext(const BatchLaunch& L, int ntiles, int grid, cudaStream_t st) {
  if (L.nb <= 0 || ntiles <= 0) return cudaSuccess;
  k_seg_ext<<<grid < ntiles ? grid : ntiles, SEG_BLOCK, 0, st>>>(batch_args(L), ntiles);
  return cudaGetLastError();
}

cudaError_t launch_seg_filter(const BatchLaunch& L, int ntiles, int grid, cudaStream_t st) {
  if (L.nb <= 0 || ntiles <= 0) return cudaSuccess;
  k_seg_filter<<<grid < ntiles ? grid : ntiles, SEG_BLOCK, 0, st>>>(batch_args(L), ntiles);
  return cudaGetLastError();
}

int batch_pad() { return 2 * Smem<512>::CHUNK + 16; }
int batch_max_instance() { return BT_MAX_CHUNKS * Smem<256>::CHUNK - 8; }

size_t batch_smem(int block) {
  return block == 512 ? sizeof(Smem<512>) : sizeof(Smem<256>);
}

cudaError_t batch_configure(int* occ256, int* occ512) {
  const void* k256[3] = {(const void*)k_batch<256, 0>, (const void*)k_batch<256, 1>, (const void*)k_batch<256, 2>};
  const void* k512[3] = {(const void*)k_batch<512, 0>, (const void*)k_batch<512, 1>, (const void*)k_batch<512, 2>};
  cudaError_t e = cudaSuccess;
  for (int m = 0; m < 3 && e == cudaSuccess; ++m) {
    e = cudaFuncSetAttribute(k256[m], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(Smem<256>));
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k512[m], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(Smem<512>));
  }
  if (e != cudaSuccess) return e;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ256, k_batch<256, 0>, 256, sizeof(Smem<256>));
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ512, k_batch<512, 0>, 512, sizeof(Smem<512>));
}

cudaError_t launch_batch(int block, int grid, const BatchLaunch& L, cudaStream_t st) {
  const BatchArgs a = batch_args(L);
  if (L.nb <= 0) return cudaSuccess;
  if (block == 512) {
    if (L.mode == 1) k_batch<512, 1><<<grid, 512, sizeof(Smem<512>), st>>>(a);
    else if (L.mode == 2) k_batch<512, 2><<<grid, 512, sizeof(Smem<512>), st>>>(a);
    else k_batch<512, 0><<<grid, 512, sizeof(Smem<512>), st>>>(a);
  } else {
    if (L.mode == 1) k_batch<256, 1><<<grid, 256, sizeof(Smem<256>), st>>>(a);
    else if (L.mode == 2) k_batch<256, 2><<<grid, 256, sizeof(Smem<256>), st>>>(a);
    else k_batch<256, 0><<<grid, 256, sizeof(Smem<256>), st>>>(a);
  }
  return cudaGetLastError();
}

cudaError_t launch_batch_output(const u32* hcount, const long long* slot0, const int* out_tmp,
                                int B, long long* out_off, int* out, long long cap, u32* error,
                                int grid, cudaStream_t st) {
  k_batch_scan<<<1, 1024, 0, st>>>(hcount, B, out_off, cap, error);
  k_batch_copy<<<grid, 256, 0, st>>>(hcount, slot0, out_tmp, out_off, B, out, cap);
  return cudaGetLastError();
}

}  // namespace gbh
