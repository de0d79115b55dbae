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
#include "filter.cuh"
#include "hull_internal.cuh"
#include "kernels.h"

namespace gbh {

namespace {

// Counts the survivors of this block's chunks (c = blockIdx.x + i * gridDim.x).
// With BULK, every whole chunk arrives by a bulk copy into a K2_STAGES-deep
// ring in shared memory, issued K2_STAGES chunks ahead; a partial last chunk
// is read directly.  A ring wait bounded by the call's spin limit that runs
// out flags ERR_TIMEOUT and counts none of the chunk's points (the call then
// reports HULL_ETIMEOUT); after it no copy is issued, and before the block
// ends every stage's last copy is waited for, so none is left in flight.
template <bool VEC, bool BULK, int K>
__device__ __forceinline__ void count_chunks(const int* __restrict__ xy, Plan* plan, u32* __restrict__ counts,
                                             unsigned char* __restrict__ mask, const Edges& E,
                                             u32* s_hist, u32* s_red, int4* ring, u64* bars, u32* s_issued,
                                             int* s_tmo) {
  const u32 n = plan->n;
  const int x0 = plan->key_x0, y0 = plan->key_y0;
  const u32 ybits = plan->ybits;
  const bool hist = plan->npasses > 0;
  const u32 spin = plan->spin_limit;
  const u32 nchunks = (n + K2_CHUNK - 1) / K2_CHUNK;
  const u32 nwhole = n / K2_CHUNK;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (BULK && threadIdx.x == 0) {
    #pragma unroll
    for (int st = 0; st < K2_STAGES; ++st) {
      const u32 c = blockIdx.x + st * gridDim.x;
      s_issued[st] = c < nwhole ? 1u : 0u;
      if (c < nwhole) k2_stage_chunk(xy, c, ring, bars, st);
    }
  }
  u32 i = 0;
  for (u32 c = blockIdx.x; c < nchunks; c += gridDim.x, ++i) {
    int px[2 * K2_PAIRS], py[2 * K2_PAIRS];
    bool keep[2 * K2_PAIRS];
    const int st = (int)(i % K2_STAGES);
    if (BULK && c < nwhole) {
      const bool ok = !*reinterpret_cast<volatile int*>(s_tmo) && mbar_wait(&bars[st], (i / K2_STAGES) & 1u, spin);
      if (ok) {
        test_staged_k<K>(ring + (size_t)st * (K2_CHUNK / 2), E, px, py, keep);
      } else {
        *s_tmo = 1;
        flag_error(plan, ERR_TIMEOUT);
        #pragma unroll
        for (int e = 0; e < 2 * K2_PAIRS; ++e) { px[e] = x0; py[e] = y0; keep[e] = false; }
      }
    } else {
      load_test_k<VEC, K>(xy, n, c * (u32)K2_CHUNK, E, px, py, keep);
    }
    u32 cnt = 0, bits = 0;
    #pragma unroll
    for (int e = 0; e < 2 * K2_PAIRS; ++e) {
      if (keep[e]) {
        ++cnt;
        bits |= 1u << e;
        if (hist) {
          const u64 key = ((u64)(u32)(px[e] - x0) << ybits) | (u64)(u32)(py[e] - y0);
          atomicAdd(&s_hist[(u32)key & (kRadix - 1)], 1u);
        }
      }
    }
    mask[(size_t)c * K2_BLOCK + threadIdx.x] = (unsigned char)bits;
    #pragma unroll
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xFFFFFFFFu, cnt, o);
    if (lane == 0) s_red[wid] = cnt;
    __syncthreads();
    if (threadIdx.x == 0) {
      u32 t = 0;
      for (int w = 0; w < K2_WARPS; ++w) t += s_red[w];
      counts[c] = t;
      // Every thread has read stage st (barrier above): refill it.
      if (BULK && !*s_tmo) {
        const u32 cn = c + K2_STAGES * gridDim.x;
        if (cn < nwhole) { k2_stage_chunk(xy, cn, ring, bars, st); ++s_issued[st]; }
      }
    }
    __syncthreads();
  }
  if (BULK && threadIdx.x == 0)
    for (int st = 0; st < K2_STAGES; ++st)
      if (s_issued[st]) mbar_wait(&bars[st], (s_issued[st] - 1u) & 1u);
}

template <bool VEC>
__global__ void __launch_bounds__(K2_BLOCK, 4)
k2_count(const int* __restrict__ xy, Plan* plan, u32* __restrict__ counts, unsigned char* __restrict__ mask) {
  extern __shared__ __align__(128) unsigned char k2_smem[];
  __shared__ u32 s_hist[kRadix];
  __shared__ u32 s_red[K2_WARPS];
  __shared__ bool s_last;
  __shared__ __align__(8) u64 s_bars[K2_STAGES];
  __shared__ u32 s_issued[K2_STAGES];
  __shared__ int s_tmo;
  int4* ring = reinterpret_cast<int4*>(k2_smem);

  if (plan->error & ERR_RANGE) return;
  const u32 n = plan->n;
  const int k = plan->ncorner;
  const bool hist = plan->npasses > 0;
  const u32 nchunks = (n + K2_CHUNK - 1) / K2_CHUNK;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  Edges E;
  load_edges(plan, k, E);
  for (int q = threadIdx.x; q < kRadix; q += K2_BLOCK) s_hist[q] = 0u;
  if (threadIdx.x == 0) s_tmo = 0;
  if (VEC && threadIdx.x == 0) {
    for (int st = 0; st < K2_STAGES; ++st) mbar_init(&s_bars[st], 1u);
    mbar_fence_init();
  }
  __syncthreads();
  switch (k) {
    case 3: count_chunks<VEC, VEC, 3>(xy, plan, counts, mask, E, s_hist, s_red, ring, s_bars, s_issued, &s_tmo); break;
    case 4: count_chunks<VEC, VEC, 4>(xy, plan, counts, mask, E, s_hist, s_red, ring, s_bars, s_issued, &s_tmo); break;
    case 5: count_chunks<VEC, VEC, 5>(xy, plan, counts, mask, E, s_hist, s_red, ring, s_bars, s_issued, &s_tmo); break;
    case 6: count_chunks<VEC, VEC, 6>(xy, plan, counts, mask, E, s_hist, s_red, ring, s_bars, s_issued, &s_tmo); break;
    case 7: count_chunks<VEC, VEC, 7>(xy, plan, counts, mask, E, s_hist, s_red, ring, s_bars, s_issued, &s_tmo); break;
    case 8: count_chunks<VEC, VEC, 8>(xy, plan, counts, mask, E, s_hist, s_red, ring, s_bars, s_issued, &s_tmo); break;
    case 9: count_chunks<VEC, VEC, 9>(xy, plan, counts, mask, E, s_hist, s_red, ring, s_bars, s_issued, &s_tmo); break;
    case 10: count_chunks<VEC, VEC, 10>(xy, plan, counts, mask, E, s_hist, s_red, ring, s_bars, s_issued, &s_tmo); break;
    case 11: count_chunks<VEC, VEC, 11>(xy, plan, counts, mask, E, s_hist, s_red, ring, s_bars, s_issued, &s_tmo); break;
    case 12: count_chunks<VEC, VEC, 12>(xy, plan, counts, mask, E, s_hist, s_red, ring, s_bars, s_issued, &s_tmo); break;
    default: count_chunks<VEC, VEC, 0>(xy, plan, counts, mask, E, s_hist, s_red, ring, s_bars, s_issued, &s_tmo); break;
  }
  if (hist)
    for (u32 q = threadIdx.x; q < kRadix; q += K2_BLOCK)
      if (s_hist[q]) atomicAdd(&plan->hist[0][q], s_hist[q]);

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
  if (threadIdx.x == K2_BLOCK - 1) plan->s = plan->s_quad = off + inc;
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

}  // namespace

int k2_tile() { return K2_CHUNK; }

cudaError_t k2_configure() {
  cudaError_t e = cudaFuncSetAttribute(k2_count<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)K2_RING_BYTES);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k2_count<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)K2_RING_BYTES);
  return e;
}

cudaError_t k2_occupancy(int* count_blocks, int* write_blocks) {
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(count_blocks, k2_count<true>, K2_BLOCK,
                                                                K2_RING_BYTES);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(write_blocks, k2_write<true>, K2_BLOCK, 0);
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
    k2_count<true><<<grid_count, K2_BLOCK, K2_RING_BYTES, st>>>(xy, plan, counts, mask);
    k2_write<true><<<grid_write, K2_BLOCK, 0, st>>>(xy, plan, counts, mask, keys_out, idx_out);
  } else {
    k2_count<false><<<grid_count, K2_BLOCK, K2_RING_BYTES, st>>>(xy, plan, counts, mask);
    k2_write<false><<<grid_write, K2_BLOCK, 0, st>>>(xy, plan, counts, mask, keys_out, idx_out);
  }
  return cudaGetLastError();
}

}  // namespace gbh
