// K2: first-round filter fused with stream compaction (Section 2.1 step 2,
// Section 3.1) and the formation of the sort key (replacing step 3's
// distance/angle with a lexicographic key).
//
// A point is discarded when it lies strictly inside the filter polygon
// (strictly left of every counter-clockwise edge, exact int64 orientation);
// with fewer than three distinct corners nothing is discarded.  Survivors
// are written as (key, idx) in ascending input order.  The compaction is
// reduce-then-scan over chunks of K2_CHUNK points, so no block ever waits
// for another:
//   k2_count  counts each chunk's survivors (and the histogram of the first
//             radix digit of their keys); the last block to finish turns
//             the counts into exclusive chunk offsets;
//   k2_write  writes each chunk's survivors (marked by k2_count in a
//             one-bit-per-point mask) at the chunk's offset, ranked by warp
//             ballots.  It walks the chunks in the reverse of k2_count's
//             order so that the most recently read part of the input is
//             still in L2.
#include "hull_internal.cuh"
#include "kernels.h"

namespace gbh {

namespace {

constexpr int K2_BLOCK = 256;
constexpr int K2_PAIRS = 4;                          // int4 loads per thread per chunk
constexpr int K2_CHUNK = K2_BLOCK * K2_PAIRS * 2;    // 2048 points
constexpr int K2_WARPS = K2_BLOCK / 32;
static_assert(K2_PAIRS * K2_WARPS == 32, "one (round, warp) count per lane");
constexpr int K2_STAGES = 3;                          // chunks in flight per block (bulk copies)
constexpr u32 K2_CHUNK_BYTES = K2_CHUNK * 2 * sizeof(int);   // 16 KB
constexpr size_t K2_RING_BYTES = (size_t)K2_STAGES * K2_CHUNK_BYTES;

// Edge j from corner c_j to c_j+1: orient(c_j, c_j+1, p) = ex*y - ey*x - c
// with c = ex*ay - ey*ax, i.e. two 32x32->64 multiply-adds per edge (every
// term is below 2^60 in magnitude for coordinates bounded by 2^29).
struct Edges {
  int ex[kMaxCorners], ney[kMaxCorners];
  long long nc[kMaxCorners];
};

template <int K>
__device__ __forceinline__ bool strictly_inside(const Edges& E, int x, int y) {
  bool in = true;
  #pragma unroll
  for (int j = 0; j < K; ++j) {
    const long long o = (long long)E.ex[j] * y + (long long)E.ney[j] * x + E.nc[j];
    in = in && (o > 0);
  }
  return in;
}

__device__ __forceinline__ void load_edges(const Plan* plan, int k, Edges& E) {
  #pragma unroll
  for (int j = 0; j < kMaxCorners; ++j) {
    const int jn = (j + 1 < k) ? j + 1 : 0;
    const int jj = (j < k) ? j : 0;
    const int ax = plan->cx[jj], ay = plan->cy[jj];
    const int ex = plan->cx[jn] - ax, ey = plan->cy[jn] - ay;
    E.ex[j] = ex;
    E.ney[j] = -ey;
    E.nc[j] = -((long long)ex * ay - (long long)ey * ax);
  }
}

// Tests this thread's pairs of a chunk against a K-corner polygon (K known
// at compile time: the corner count is uniform over the whole launch).
template <bool VEC, int K>
__device__ __forceinline__ void load_test_k(const int* __restrict__ xy, u32 n, u32 base,
                                            const Edges& E, int* px, int* py, bool* keep) {
  #pragma unroll
  for (int r = 0; r < K2_PAIRS; ++r) {
    const u32 i0 = base + 2u * (r * K2_BLOCK + threadIdx.x);
    if (VEC && i0 + 1 < n) {
      const int4 v = *reinterpret_cast<const int4*>(xy + 2 * (size_t)i0);
      px[2 * r] = v.x; py[2 * r] = v.y; px[2 * r + 1] = v.z; py[2 * r + 1] = v.w;
    } else {
      int2 a = make_int2(0, 0), b = make_int2(0, 0);
      if (i0 < n) a = *reinterpret_cast<const int2*>(xy + 2 * (size_t)i0);
      if (i0 + 1 < n) b = *reinterpret_cast<const int2*>(xy + 2 * (size_t)i0 + 2);
      px[2 * r] = a.x; py[2 * r] = a.y; px[2 * r + 1] = b.x; py[2 * r + 1] = b.y;
    }
    keep[2 * r] = (i0 < n) && !(K >= 3 && strictly_inside<K>(E, px[2 * r], py[2 * r]));
    keep[2 * r + 1] = (i0 + 1 < n) && !(K >= 3 && strictly_inside<K>(E, px[2 * r + 1], py[2 * r + 1]));
  }
}

// Tests this thread's pairs of a chunk staged in shared memory.
template <int K>
__device__ __forceinline__ void test_staged_k(const int4* __restrict__ chunk, const Edges& E,
                                              int* px, int* py, bool* keep) {
  #pragma unroll
  for (int r = 0; r < K2_PAIRS; ++r) {
    const int4 v = chunk[r * K2_BLOCK + threadIdx.x];
    px[2 * r] = v.x; py[2 * r] = v.y; px[2 * r + 1] = v.z; py[2 * r + 1] = v.w;
    keep[2 * r] = !(K >= 3 && strictly_inside<K>(E, v.x, v.y));
    keep[2 * r + 1] = !(K >= 3 && strictly_inside<K>(E, v.z, v.w));
  }
}

// Issues the bulk copy of chunk c into ring stage st (one thread).
__device__ __forceinline__ void k2_stage_chunk(const int* xy, u32 c, int4* ring, u64* bars, int st) {
  mbar_arrive_expect_tx(&bars[st], K2_CHUNK_BYTES);
  bulk_load(ring + (size_t)st * (K2_CHUNK / 2), xy + (size_t)c * 2 * K2_CHUNK, K2_CHUNK_BYTES, &bars[st]);
}

// Counts the survivors of this block's chunks (c = blockIdx.x + i * gridDim.x).
// With BULK, every whole chunk arrives by a bulk copy into a K2_STAGES-deep
// ring in shared memory, issued K2_STAGES chunks ahead; a partial last chunk
// is read directly.
template <bool VEC, bool BULK, bool BINS, int K>
__device__ __forceinline__ void count_chunks(const int* __restrict__ xy, Plan* plan, u32* __restrict__ counts,
                                             unsigned char* __restrict__ mask, const Edges& E,
                                             u32* s_hist, u32* s_red, int4* ring, u64* bars, u32* s_bins) {
  const u32 n = plan->n;
  const int x0 = plan->key_x0, y0 = plan->key_y0;
  const u32 ybits = plan->ybits;
  const u32 fshift = plan->fshift;
  const bool hist = !BINS && plan->npasses > 0;
  const u32 nchunks = (n + K2_CHUNK - 1) / K2_CHUNK;
  const u32 nwhole = n / K2_CHUNK;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (BULK && threadIdx.x == 0) {
    #pragma unroll
    for (int st = 0; st < K2_STAGES; ++st) {
      const u32 c = blockIdx.x + st * gridDim.x;
      if (c < nwhole) k2_stage_chunk(xy, c, ring, bars, st);
    }
  }
  u32 i = 0;
  for (u32 c = blockIdx.x; c < nchunks; c += gridDim.x, ++i) {
    int px[2 * K2_PAIRS], py[2 * K2_PAIRS];
    bool keep[2 * K2_PAIRS];
    const int st = (int)(i % K2_STAGES);
    if (BULK && c < nwhole) {
      if (!mbar_wait(&bars[st], (i / K2_STAGES) & 1u)) flag_error(plan, ERR_TIMEOUT);
      test_staged_k<K>(ring + (size_t)st * (K2_CHUNK / 2), E, px, py, keep);
    } else {
      load_test_k<VEC, K>(xy, n, c * (u32)K2_CHUNK, E, px, py, keep);
    }
    u32 cnt = 0, bits = 0;
    #pragma unroll
    for (int e = 0; e < 2 * K2_PAIRS; ++e) {
      if (keep[e]) {
        ++cnt;
        bits |= 1u << e;
        if (hist || BINS) {
          const u64 key = ((u64)(u32)(px[e] - x0) << ybits) | (u64)(u32)(py[e] - y0);
          if (BINS) atomicAdd(&s_bins[(u32)(key >> fshift)], 1u);
          else atomicAdd(&s_hist[(u32)key & (kRadix - 1)], 1u);
        }
      }
    }
    mask[(size_t)c * K2_BLOCK + threadIdx.x] = (unsigned char)bits;
    if (!BINS) {          // chunk counts for the stable compaction (the bin rows replace them)
      #pragma unroll
      for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xFFFFFFFFu, cnt, o);
      if (lane == 0) s_red[wid] = cnt;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      if (!BINS) {
        u32 t = 0;
        for (int w = 0; w < K2_WARPS; ++w) t += s_red[w];
        counts[c] = t;
      }
      // Every thread has read stage st (barrier above): refill it.
      if (BULK) {
        const u32 cn = c + K2_STAGES * gridDim.x;
        if (cn < nwhole) k2_stage_chunk(xy, cn, ring, bars, st);
      }
    }
    __syncthreads();
  }
}

// With BINS, also counts the survivors per bin of the bucket sort (key >>
// fshift; dynamic shared memory: the ring, then kBins counters), adds them
// to the bins' totals btot, and reserves the block's run in every coarse
// bin (kFinePerCoarse consecutive bins) from the coarse cursors ccur: row
// blockIdx.x of `rows` (kCoarse words) receives the run's offset in its
// coarse bin.  btot and ccur start at zero.
template <bool VEC, bool BINS>
__global__ void __launch_bounds__(K2_BLOCK, 4)
k2_count(const int* __restrict__ xy, Plan* plan, u32* __restrict__ counts,
         unsigned char* __restrict__ mask, u32* __restrict__ rows, u32* __restrict__ btot,
         u32* __restrict__ ccur) {
  extern __shared__ __align__(128) unsigned char k2_smem[];
  __shared__ u32 s_hist[kRadix];
  __shared__ u32 s_red[K2_WARPS];
  __shared__ bool s_last;
  __shared__ __align__(8) u64 s_bars[K2_STAGES];
  int4* ring = reinterpret_cast<int4*>(k2_smem);
  u32* s_bins = reinterpret_cast<u32*>(k2_smem + K2_RING_BYTES);

  if (plan->error & ERR_RANGE) return;
  const u32 n = plan->n;
  const int k = plan->ncorner;
  const bool hist = !BINS && plan->npasses > 0;
  const u32 nchunks = (n + K2_CHUNK - 1) / K2_CHUNK;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  Edges E;
  load_edges(plan, k, E);
  for (int q = threadIdx.x; q < kRadix; q += K2_BLOCK) s_hist[q] = 0u;
  if (BINS)
    for (int q = threadIdx.x; q < kBins; q += K2_BLOCK) s_bins[q] = 0u;
  if (VEC && threadIdx.x == 0) {
    for (int st = 0; st < K2_STAGES; ++st) mbar_init(&s_bars[st], 1u);
    mbar_fence_init();
  }
  __syncthreads();
  switch (k) {
    case 3: count_chunks<VEC, VEC, BINS, 3>(xy, plan, counts, mask, E, s_hist, s_red, ring, s_bars, s_bins); break;
    case 4: count_chunks<VEC, VEC, BINS, 4>(xy, plan, counts, mask, E, s_hist, s_red, ring, s_bars, s_bins); break;
    case 5: count_chunks<VEC, VEC, BINS, 5>(xy, plan, counts, mask, E, s_hist, s_red, ring, s_bars, s_bins); break;
    case 6: count_chunks<VEC, VEC, BINS, 6>(xy, plan, counts, mask, E, s_hist, s_red, ring, s_bars, s_bins); break;
    case 7: count_chunks<VEC, VEC, BINS, 7>(xy, plan, counts, mask, E, s_hist, s_red, ring, s_bars, s_bins); break;
    case 8: count_chunks<VEC, VEC, BINS, 8>(xy, plan, counts, mask, E, s_hist, s_red, ring, s_bars, s_bins); break;
    case 9: count_chunks<VEC, VEC, BINS, 9>(xy, plan, counts, mask, E, s_hist, s_red, ring, s_bars, s_bins); break;
    case 10: count_chunks<VEC, VEC, BINS, 10>(xy, plan, counts, mask, E, s_hist, s_red, ring, s_bars, s_bins); break;
    case 11: count_chunks<VEC, VEC, BINS, 11>(xy, plan, counts, mask, E, s_hist, s_red, ring, s_bars, s_bins); break;
    case 12: count_chunks<VEC, VEC, BINS, 12>(xy, plan, counts, mask, E, s_hist, s_red, ring, s_bars, s_bins); break;
    default: count_chunks<VEC, VEC, BINS, 0>(xy, plan, counts, mask, E, s_hist, s_red, ring, s_bars, s_bins); break;
  }
  if (hist)
    for (u32 q = threadIdx.x; q < kRadix; q += K2_BLOCK)
      if (s_hist[q]) atomicAdd(&plan->hist[0][q], s_hist[q]);
  if (BINS) {
    // k_binstart turns the totals into bin starts and sets the survivor count.
    __syncthreads();
    for (u32 q = threadIdx.x; q < (u32)kBins; q += K2_BLOCK) {
      const u32 v = s_bins[q];
      if (v) atomicAdd(&btot[q], v);
    }
    for (u32 cb = threadIdx.x; cb < (u32)kCoarse; cb += K2_BLOCK) {
      u32 cs = 0;
      #pragma unroll 8
      for (u32 f = 0; f < (u32)kFinePerCoarse; ++f) cs += s_bins[cb * kFinePerCoarse + ((f + cb) & (kFinePerCoarse - 1))];
      rows[(size_t)blockIdx.x * kCoarse + cb] = cs ? atomicAdd(&ccur[cb], cs) : 0u;
    }
    return;
  }

  // The last block turns the chunk counts into exclusive offsets.
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(&plan->ctr[CTR_FILTER], 1u) == gridDim.x - 1;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  const u32 per = (nchunks + K2_BLOCK - 1) / K2_BLOCK;
  const u32 lo = min(nchunks, threadIdx.x * per), hi = min(nchunks, lo + per);
  u32 sum = 0;
  for (u32 c = lo; c < hi; ++c) sum += *reinterpret_cast<volatile u32*>(&counts[c]);
  u32 inc = sum;
  #pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const u32 t = __shfl_up_sync(0xFFFFFFFFu, inc, o);
    if (lane >= o) inc += t;
  }
  if (lane == 31) s_red[wid] = inc;
  __syncthreads();
  u32 off = 0;
  for (int w = 0; w < wid; ++w) off += s_red[w];
  u32 run = off + inc - sum;
  for (u32 c = lo; c < hi; ++c) {
    const u32 v = *reinterpret_cast<volatile u32*>(&counts[c]);
    counts[c] = run;
    run += v;
  }
  if (threadIdx.x == K2_BLOCK - 1) plan->s = off + inc;
}

template <bool VEC>
__global__ void __launch_bounds__(K2_BLOCK, 6)
k2_write(const int* __restrict__ xy, Plan* plan, const u32* __restrict__ offsets,
         const unsigned char* __restrict__ mask, u64* __restrict__ keys_out,
         u32* __restrict__ idx_out) {
  __shared__ u32 s_wcnt[K2_PAIRS * K2_WARPS];

  if (plan->error & ERR_RANGE) return;
  const u32 n = plan->n;
  const u32 s = plan->s;
  const int k = plan->ncorner;
  const int x0 = plan->key_x0, y0 = plan->key_y0;
  const u32 ybits = plan->ybits;
  const u32 nchunks = (n + K2_CHUNK - 1) / K2_CHUNK;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const u32 lt_mask = (1u << lane) - 1u;
  (void)k;

  for (u32 q = blockIdx.x; q < nchunks; q += gridDim.x) {
    const u32 c = nchunks - 1 - q;
    const u32 base = c * (u32)K2_CHUNK;
    const u32 bits = mask[(size_t)c * K2_BLOCK + threadIdx.x];
    int px[2 * K2_PAIRS], py[2 * K2_PAIRS];
    bool keep[2 * K2_PAIRS];
    #pragma unroll
    for (int r = 0; r < K2_PAIRS; ++r) {
      const u32 i0 = base + 2u * (r * K2_BLOCK + threadIdx.x);
      keep[2 * r] = (bits >> (2 * r)) & 1u;
      keep[2 * r + 1] = (bits >> (2 * r + 1)) & 1u;
      if (VEC && i0 + 1 < n) {
        if (keep[2 * r] | keep[2 * r + 1]) {
          const int4 v = *reinterpret_cast<const int4*>(xy + 2 * (size_t)i0);
          px[2 * r] = v.x; py[2 * r] = v.y; px[2 * r + 1] = v.z; py[2 * r + 1] = v.w;
        } else {
          px[2 * r] = py[2 * r] = px[2 * r + 1] = py[2 * r + 1] = 0;
        }
      } else {
        int2 a = make_int2(0, 0), b = make_int2(0, 0);
        if (i0 < n) a = *reinterpret_cast<const int2*>(xy + 2 * (size_t)i0);
        if (i0 + 1 < n) b = *reinterpret_cast<const int2*>(xy + 2 * (size_t)i0 + 2);
        px[2 * r] = a.x; py[2 * r] = a.y; px[2 * r + 1] = b.x; py[2 * r + 1] = b.y;
      }
    }
    // Ranks in (round, warp, lane, element) order, which is input order.
    u32 lane_pre[K2_PAIRS];
    #pragma unroll
    for (int r = 0; r < K2_PAIRS; ++r) {
      const u32 b0 = __ballot_sync(0xFFFFFFFFu, keep[2 * r]);
      const u32 b1 = __ballot_sync(0xFFFFFFFFu, keep[2 * r + 1]);
      lane_pre[r] = __popc(b0 & lt_mask) + __popc(b1 & lt_mask);
      if (lane == 0) s_wcnt[r * K2_WARPS + wid] = __popc(b0) + __popc(b1);
    }
    __syncthreads();
    if (wid == 0) {
      const u32 c0 = s_wcnt[lane];
      u32 inc = c0;
      #pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const u32 t = __shfl_up_sync(0xFFFFFFFFu, inc, o);
        if (lane >= o) inc += t;
      }
      s_wcnt[lane] = inc - c0;
    }
    __syncthreads();
    const u32 excl = offsets[c];
    #pragma unroll
    for (int r = 0; r < K2_PAIRS; ++r) {
      u32 pos = excl + s_wcnt[r * K2_WARPS + wid] + lane_pre[r];
      const u32 i0 = base + 2u * (r * K2_BLOCK + threadIdx.x);
      #pragma unroll
      for (int e = 0; e < 2; ++e) {
        if (keep[2 * r + e]) {
          if (pos < s) {
            keys_out[pos] = ((u64)(u32)(px[2 * r + e] - x0) << ybits) | (u64)(u32)(py[2 * r + e] - y0);
            idx_out[pos] = i0 + e;
          } else {
            flag_error(plan, ERR_INTERNAL);
          }
          ++pos;
        }
      }
    }
    __syncthreads();
  }
}

// The bucket sort's first scatter: writes every survivor (marked by
// k2_count in `mask`) as (key, index) into its coarse bin (kCoarse of them,
// each the union of kFinePerCoarse consecutive bins).  Block i walks the
// same chunks as block i of k2_count (in the reverse order, so that the part
// of the input k2_count read last is still in L2); its run in coarse bin c
// starts at bstart of c's first bin plus the offset k2_count reserved for
// block i in c (rows[i][c]), and grows one survivor at a time
// (positions by shared-memory atomics, in no particular order), so every
// block has only one partly written sector per coarse bin at a time and L2
// completes it before it leaves.  No block waits for another.  Whole chunks
// and their mask bytes arrive by bulk copies into a K2_STAGES-deep ring
// (evict-first: nothing reads the input again); the stores are marked
// evict-last.  k3_split then spreads every coarse bin over its bins.
constexpr u32 K2_MASK_BYTES = K2_BLOCK;                    // one byte per thread and chunk
constexpr u32 K2_SC_STAGE = K2_CHUNK_BYTES + K2_MASK_BYTES;

__device__ __forceinline__ void k2_sc_stage(const int* xy, const unsigned char* mask, u32 c, unsigned char* ring,
                                            u64* bars, int st, u64 pol) {
  unsigned char* dst = ring + (size_t)st * K2_SC_STAGE;
  mbar_arrive_expect_tx(&bars[st], K2_SC_STAGE);
  bulk_load_hint(dst, xy + (size_t)c * 2 * K2_CHUNK, K2_CHUNK_BYTES, &bars[st], pol);
  bulk_load_hint(dst + K2_CHUNK_BYTES, mask + (size_t)c * K2_BLOCK, K2_MASK_BYTES, &bars[st], pol);
}

// Shared memory of k2_scatter after the ring: the chunk's survivors in
// coarse-bin order, and per coarse bin the block's cursor, the chunk's
// count, first staging slot and first global position.
struct K2ScatterSmem {
  u64 key[K2_CHUNK];
  u32 idx[K2_CHUNK];
  u32 cur[kCoarse];
  u32 cnt[kCoarse];
  u32 lst[kCoarse];
  u32 gb[kCoarse];
  u32 wsum[K2_WARPS];
};
constexpr size_t K2_SC_SMEM = (size_t)K2_STAGES * K2_SC_STAGE + sizeof(K2ScatterSmem);
static_assert(kCoarse == K2_BLOCK, "one thread per coarse bin");

// Scatters the kept points of chunk c (this thread's keep bits `bits` and
// points px/py in its pair order; every thread of the block calls it):
// ranks within the chunk per coarse bin, one reservation per coarse bin on
// the block's cursor, the chunk staged in coarse-bin order, then written
// with consecutive threads on consecutive positions.
__device__ __forceinline__ void k2_scatter_chunk(Plan* plan, u32 c, u32 bits, const int* px, const int* py, int x0,
                                                 int y0, u32 ybits, u32 cshift, u32 s, K2ScatterSmem& S,
                                                 u64* keys_out, u32* idx_out, u64 pol) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const u32 base = c * (u32)K2_CHUNK;
  u64 key[2 * K2_PAIRS];
  u32 rk[2 * K2_PAIRS];
  #pragma unroll
  for (int e = 0; e < 2 * K2_PAIRS; ++e) {
    key[e] = ((u64)(u32)(px[e] - x0) << ybits) | (u64)(u32)(py[e] - y0);
    rk[e] = ((bits >> e) & 1u) ? atomicAdd(&S.cnt[(u32)(key[e] >> cshift)], 1u) : 0xFFFFFFFFu;
  }
  __syncthreads();
  {
    const u32 cb = threadIdx.x;                      // this thread's coarse bin
    const u32 n = S.cnt[cb];
    u32 inc = n;
    #pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const u32 t = __shfl_up_sync(0xFFFFFFFFu, inc, o);
      if (lane >= o) inc += t;
    }
    if (lane == 31) S.wsum[wid] = inc;
    __syncthreads();
    u32 off = inc - n;
    for (int w = 0; w < wid; ++w) off += S.wsum[w];
    S.lst[cb] = off;
    S.gb[cb] = S.cur[cb];
    S.cur[cb] += n;
  }
  __syncthreads();
  u32 total = 0;
  for (int w = 0; w < K2_WARPS; ++w) total += S.wsum[w];
  #pragma unroll
  for (int e = 0; e < 2 * K2_PAIRS; ++e) {
    if (rk[e] != 0xFFFFFFFFu) {
      const u32 p = S.lst[(u32)(key[e] >> cshift)] + rk[e];
      S.key[p] = key[e];
      S.idx[p] = base + 2u * ((e >> 1) * K2_BLOCK + threadIdx.x) + (u32)(e & 1);
    }
  }
  __syncthreads();
  for (u32 j = threadIdx.x; j < total; j += K2_BLOCK) {
    const u64 k = S.key[j];
    const u32 cb = (u32)(k >> cshift);
    const u32 pos = S.gb[cb] + (j - S.lst[cb]);
    if (pos < s) {
      st_hint_u64(keys_out + pos, k, pol);
      st_hint_u32(idx_out + pos, S.idx[j], pol);
    } else {
      flag_error(plan, ERR_INTERNAL);
    }
  }
  S.cnt[threadIdx.x] = 0u;          // read by everyone before the barrier above
  __syncthreads();
}

template <bool VEC>
__global__ void __launch_bounds__(K2_BLOCK, 2)
k2_scatter(const int* __restrict__ xy, Plan* plan, const unsigned char* __restrict__ mask,
           const u32* __restrict__ rows, const u32* __restrict__ bstart, u64* __restrict__ keys_out,
           u32* __restrict__ idx_out) {
  extern __shared__ __align__(128) unsigned char k2s_smem[];
  __shared__ __align__(8) u64 s_bars[K2_STAGES];
  unsigned char* ring = k2s_smem;
  K2ScatterSmem& S = *reinterpret_cast<K2ScatterSmem*>(k2s_smem + (size_t)K2_STAGES * K2_SC_STAGE);
  if (plan->error & ERR_RANGE) return;
  const u32 n = plan->n;
  const u32 s = plan->s;
  const int x0 = plan->key_x0, y0 = plan->key_y0;
  const u32 ybits = plan->ybits;
  const u32 cshift = plan->fshift + (u32)(kBinBits - kCoarseBits);
  const u32 nchunks = (n + K2_CHUNK - 1) / K2_CHUNK;
  const u32 G = gridDim.x, b0 = blockIdx.x;
  const u64 pol_in = policy_evict_first();
  const u64 pol_out = policy_evict_last();
  {
    const u32 cb = threadIdx.x;
    S.cur[cb] = bstart[cb * kFinePerCoarse] + rows[(size_t)b0 * kCoarse + cb];
    S.cnt[cb] = 0u;
  }
  // This block's chunks are b0 + k * G.  The whole ones (c < nring) go
  // through the ring, last first; the rest are read directly.
  const u32 nring = VEC ? n / K2_CHUNK : 0u;
  const u32 kw = b0 < nring ? (nring - 1 - b0) / G + 1 : 0u;
  const u32 kall = b0 < nchunks ? (nchunks - 1 - b0) / G + 1 : 0u;
  auto ring_chunk = [&](u32 q) { return b0 + (kw - 1 - q) * G; };
  if (VEC && threadIdx.x == 0) {
    for (int st = 0; st < K2_STAGES; ++st) mbar_init(&s_bars[st], 1u);
    mbar_fence_init();
  }
  __syncthreads();
  if (VEC && threadIdx.x == 0)
    for (u32 q = 0; q < (u32)K2_STAGES && q < kw; ++q)
      k2_sc_stage(xy, mask, ring_chunk(q), ring, s_bars, (int)q, pol_in);
  for (u32 q = 0; q < kw; ++q) {
    const int st = (int)(q % K2_STAGES);
    if (!mbar_wait(&s_bars[st], (q / K2_STAGES) & 1u)) flag_error(plan, ERR_TIMEOUT);
    const unsigned char* stage = ring + (size_t)st * K2_SC_STAGE;
    const u32 bits = stage[K2_CHUNK_BYTES + threadIdx.x];
    const int4* pts = reinterpret_cast<const int4*>(stage);
    int px[2 * K2_PAIRS], py[2 * K2_PAIRS];
    #pragma unroll
    for (int r = 0; r < K2_PAIRS; ++r) {
      const int4 v = pts[r * K2_BLOCK + threadIdx.x];
      px[2 * r] = v.x; py[2 * r] = v.y; px[2 * r + 1] = v.z; py[2 * r + 1] = v.w;
    }
    // Every thread has read stage st (the chunk's first barrier follows).
    k2_scatter_chunk(plan, ring_chunk(q), bits, px, py, x0, y0, ybits, cshift, s, S, keys_out, idx_out, pol_out);
    if (threadIdx.x == 0 && q + K2_STAGES < kw)
      k2_sc_stage(xy, mask, ring_chunk(q + K2_STAGES), ring, s_bars, st, pol_in);
  }
  for (u32 k = kw; k < kall; ++k) {
    const u32 c = b0 + k * G;
    const u32 base = c * (u32)K2_CHUNK;
    const u32 bits = mask[(size_t)c * K2_BLOCK + threadIdx.x];
    int px[2 * K2_PAIRS], py[2 * K2_PAIRS];
    #pragma unroll
    for (int r = 0; r < K2_PAIRS; ++r) {
      const u32 i0 = base + 2u * (r * K2_BLOCK + threadIdx.x);
      int2 a = make_int2(0, 0), b = make_int2(0, 0);
      if ((bits >> (2 * r)) & 1u) a = *reinterpret_cast<const int2*>(xy + 2 * (size_t)i0);
      if ((bits >> (2 * r + 1)) & 1u) b = *reinterpret_cast<const int2*>(xy + 2 * (size_t)i0 + 2);
      px[2 * r] = a.x; py[2 * r] = a.y; px[2 * r + 1] = b.x; py[2 * r + 1] = b.y;
    }
    k2_scatter_chunk(plan, c, bits, px, py, x0, y0, ybits, cshift, s, S, keys_out, idx_out, pol_out);
  }
}

}  // namespace

int k2_tile() { return K2_CHUNK; }

constexpr size_t K2_BINS_SMEM = K2_RING_BYTES + (size_t)kBins * sizeof(u32);

cudaError_t k2_configure() {
  cudaError_t e = cudaFuncSetAttribute(k2_count<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)K2_RING_BYTES);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k2_count<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)K2_RING_BYTES);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k2_count<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)K2_BINS_SMEM);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k2_count<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)K2_BINS_SMEM);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k2_scatter<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)K2_SC_SMEM);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k2_scatter<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)K2_SC_SMEM);
  return e;
}

cudaError_t k2_occupancy(int* count_blocks, int* write_blocks) {
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(count_blocks, k2_count<true, false>, K2_BLOCK,
                                                                K2_RING_BYTES);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(write_blocks, k2_write<true>, K2_BLOCK, 0);
  return e;
}

cudaError_t k2_bins_occupancy(int* blocks) {
  int a = 0, b = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k2_count<true, true>, K2_BLOCK, K2_BINS_SMEM);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k2_scatter<true>, K2_BLOCK, K2_SC_SMEM);
  *blocks = a < b ? a : b;
  return e;
}

// `status` holds one 32-bit count (then offset) per chunk; `mask` one byte
// per thread and chunk (n / 8 bytes, rounded up to whole chunks).
// A 16-byte aligned input is counted through bulk copies (the ring is
// allocated either way, so both instances share one occupancy).
cudaError_t launch_k2(const int* xy, Plan* plan, u64* keys_out, u32* idx_out, u64* status,
                      unsigned char* mask, int grid_count, int grid_write, cudaStream_t st) {
  const bool vec = (reinterpret_cast<uintptr_t>(xy) & 15u) == 0;
  u32* counts = reinterpret_cast<u32*>(status);
  if (vec) {
    k2_count<true, false><<<grid_count, K2_BLOCK, K2_RING_BYTES, st>>>(xy, plan, counts, mask, nullptr, nullptr, nullptr);
    k2_write<true><<<grid_write, K2_BLOCK, 0, st>>>(xy, plan, counts, mask, keys_out, idx_out);
  } else {
    k2_count<false, false><<<grid_count, K2_BLOCK, K2_RING_BYTES, st>>>(xy, plan, counts, mask, nullptr, nullptr, nullptr);
    k2_write<false><<<grid_write, K2_BLOCK, 0, st>>>(xy, plan, counts, mask, keys_out, idx_out);
  }
  return cudaGetLastError();
}

// First round for the bucket sort: k2_count with the bins' totals and every
// block's coarse-bin offsets (rows: grid rows of kCoarse words; bcnt: kBins
// totals then kCoarse cursors, cleared here), then the bin starts and groups
// (k3_bucket.cu); launch_k2_bins_scatter then writes the survivors into
// their coarse bins with the same `grid` (the scatter walks the count's
// chunks).
cudaError_t launch_k2_bins(const int* xy, Plan* plan, u64* status, unsigned char* mask, u32* rows, u32* bcnt,
                           u32* bstart, uint2* groups, u32* fcur, int grid, cudaStream_t st) {
  const bool vec = (reinterpret_cast<uintptr_t>(xy) & 15u) == 0;
  u32* counts = reinterpret_cast<u32*>(status);
  u32* btot = bcnt;
  u32* ccur = bcnt + kBins;
  cudaError_t e = cudaMemsetAsync(bcnt, 0, ((size_t)kBins + kCoarse) * sizeof(u32), st);
  if (e != cudaSuccess) return e;
  if (vec) k2_count<true, true><<<grid, K2_BLOCK, K2_BINS_SMEM, st>>>(xy, plan, counts, mask, rows, btot, ccur);
  else k2_count<false, true><<<grid, K2_BLOCK, K2_BINS_SMEM, st>>>(xy, plan, counts, mask, rows, btot, ccur);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_binstart(btot, plan, bstart, groups, fcur, st);
}

cudaError_t launch_k2_bins_scatter(const int* xy, Plan* plan, u64* keys_out, u32* idx_out, const unsigned char* mask,
                                   const u32* rows, const u32* bstart, int grid, cudaStream_t st) {
  const bool vec = (reinterpret_cast<uintptr_t>(xy) & 15u) == 0;
  if (vec) k2_scatter<true><<<grid, K2_BLOCK, K2_SC_SMEM, st>>>(xy, plan, mask, rows, bstart, keys_out, idx_out);
  else k2_scatter<false><<<grid, K2_BLOCK, K2_SC_SMEM, st>>>(xy, plan, mask, rows, bstart, keys_out, idx_out);
  return cudaGetLastError();
}

}  // namespace gbh
