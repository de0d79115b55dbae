// K2: first-round filter fused with stream compaction (Section 2.1 step 2,
// Section 3.1) and the formation of the sort key (replacing step 3's
// distance/angle with a lexicographic key).
//
// A point is discarded when it lies strictly inside the filter polygon
// (strictly left of every counter-clockwise edge, exact int64 orientation);
// with fewer than three distinct corners nothing is discarded.  Survivors
// are written as (key, idx) in ascending input order: warp ballots give the
// ranks inside a tile and one decoupled look-back over tiles (dynamic tile
// ids, so every awaited tile belongs to a running block) gives the tile's
// output offset.  The digit histograms of the survivors' keys, needed by
// every radix pass, are accumulated here as well, so the sort needs no
// separate histogram pass.
#include "hull_internal.cuh"
#include "kernels.h"

namespace gbh {

namespace {

constexpr int K2_BLOCK = 256;
constexpr int K2_PAIRS = 8;                          // int4 loads per thread per tile
constexpr int K2_TILE = K2_BLOCK * K2_PAIRS * 2;     // 4096 points
constexpr int K2_WARPS = K2_BLOCK / 32;

struct Edges {
  int ax[kMaxCorners], ay[kMaxCorners], ex[kMaxCorners], ey[kMaxCorners];
};

template <int K>
__device__ __forceinline__ bool strictly_inside(const Edges& E, int x, int y) {
  bool in = true;
  #pragma unroll
  for (int j = 0; j < K; ++j) {
    long long o = (long long)E.ex[j] * (y - E.ay[j]) - (long long)E.ey[j] * (x - E.ax[j]);
    in = in && (o > 0);
  }
  return in;
}

__device__ __forceinline__ bool inside_any(const Edges& E, int k, int x, int y) {
  switch (k) {
    case 3: return strictly_inside<3>(E, x, y);
    case 4: return strictly_inside<4>(E, x, y);
    case 5: return strictly_inside<5>(E, x, y);
    case 6: return strictly_inside<6>(E, x, y);
    case 7: return strictly_inside<7>(E, x, y);
    case 8: return strictly_inside<8>(E, x, y);
    default: return false;
  }
}

template <bool VEC>
__global__ void __launch_bounds__(K2_BLOCK)
k2_filter(const int* __restrict__ xy, Plan* plan, u64* __restrict__ keys_out,
          u32* __restrict__ idx_out, u64* __restrict__ status) {
  __shared__ u32 s_hist[kMaxPasses * kRadix];
  __shared__ u32 s_wcnt[K2_PAIRS * K2_WARPS];
  __shared__ u32 s_excl;
  __shared__ u32 s_tile;
  __shared__ int s_fail;

  if (plan->error & ERR_RANGE) return;
  const u32 n = plan->n;
  const int k = plan->ncorner;
  const u32 epoch = plan->epoch + EP_FILTER;
  const u32 spin = plan->spin_limit;
  const int x0 = plan->key_x0, y0 = plan->key_y0;
  const u32 ybits = plan->ybits;
  const u32 npasses = plan->npasses;
  const u32 ntiles = (n + K2_TILE - 1) / K2_TILE;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const u32 lt_mask = (1u << lane) - 1u;

  Edges E;
  #pragma unroll
  for (int j = 0; j < kMaxCorners; ++j) {
    int jn = (j + 1 < k) ? j + 1 : 0;
    int jj = (j < k) ? j : 0;
    E.ax[j] = plan->cx[jj];
    E.ay[j] = plan->cy[jj];
    E.ex[j] = plan->cx[jn] - plan->cx[jj];
    E.ey[j] = plan->cy[jn] - plan->cy[jj];
  }
  for (int q = threadIdx.x; q < kMaxPasses * kRadix; q += K2_BLOCK) s_hist[q] = 0u;

  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) s_tile = atomicAdd(&plan->ctr[CTR_FILTER], 1u);
    __syncthreads();
    const u32 tile = s_tile;
    if (tile >= ntiles) break;
    const u32 base = tile * (u32)K2_TILE;

    int px[2 * K2_PAIRS], py[2 * K2_PAIRS];
    bool keep[2 * K2_PAIRS];
    #pragma unroll
    for (int r = 0; r < K2_PAIRS; ++r) {
      const u32 i0 = base + 2u * (r * K2_BLOCK + threadIdx.x);
      if (VEC && i0 + 1 < n) {
        int4 v = *reinterpret_cast<const int4*>(xy + 2 * (size_t)i0);
        px[2 * r] = v.x; py[2 * r] = v.y; px[2 * r + 1] = v.z; py[2 * r + 1] = v.w;
      } else {
        int2 a = make_int2(0, 0), b = make_int2(0, 0);
        if (i0 < n) a = *reinterpret_cast<const int2*>(xy + 2 * (size_t)i0);
        if (i0 + 1 < n) b = *reinterpret_cast<const int2*>(xy + 2 * (size_t)i0 + 2);
        px[2 * r] = a.x; py[2 * r] = a.y; px[2 * r + 1] = b.x; py[2 * r + 1] = b.y;
      }
      keep[2 * r] = (i0 < n) && !inside_any(E, k, px[2 * r], py[2 * r]);
      keep[2 * r + 1] = (i0 + 1 < n) && !inside_any(E, k, px[2 * r + 1], py[2 * r + 1]);
    }

    // Ranks in (round, warp, lane, element) order, which is input order.
    u32 lane_pre[K2_PAIRS];
    #pragma unroll
    for (int r = 0; r < K2_PAIRS; ++r) {
      u32 b0 = __ballot_sync(0xFFFFFFFFu, keep[2 * r]);
      u32 b1 = __ballot_sync(0xFFFFFFFFu, keep[2 * r + 1]);
      lane_pre[r] = __popc(b0 & lt_mask) + __popc(b1 & lt_mask);
      if (lane == 0) s_wcnt[r * K2_WARPS + wid] = __popc(b0) + __popc(b1);
    }
    // Digit histograms of the survivors' keys for every radix pass.
    #pragma unroll
    for (int e = 0; e < 2 * K2_PAIRS; ++e) {
      if (keep[e]) {
        u64 key = ((u64)(u32)(px[e] - x0) << ybits) | (u64)(u32)(py[e] - y0);
        for (u32 p = 0; p < npasses; ++p)
          atomicAdd(&s_hist[p * kRadix + (u32)((key >> (p * kRadixBits)) & (kRadix - 1))], 1u);
      }
    }
    __syncthreads();
    if (wid == 0) {
      // Exclusive scan of the 64 (round, warp) counts, two per lane.
      u32 c0 = s_wcnt[2 * lane], c1 = s_wcnt[2 * lane + 1];
      u32 sum = c0 + c1, inc = sum;
      #pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        u32 t = __shfl_up_sync(0xFFFFFFFFu, inc, o);
        if (lane >= o) inc += t;
      }
      u32 ex = inc - sum;
      s_wcnt[2 * lane] = ex;
      s_wcnt[2 * lane + 1] = ex + c0;
      const u32 total = __shfl_sync(0xFFFFFFFFu, inc, 31);
      u32 excl = 0;
      bool failed = false;
      if (tile == 0) {
        if (lane == 0) st_release_u64(&status[0], make_status(epoch, ST_INCL, total));
      } else {
        if (lane == 0) st_release_u64(&status[tile], make_status(epoch, ST_AGG, total));
        excl = warp_lookback_count(status, tile, epoch, plan, spin, &failed);
        if (lane == 0 && !failed) st_release_u64(&status[tile], make_status(epoch, ST_INCL, excl + total));
      }
      if (lane == 0) {
        s_excl = excl;
        s_fail = failed ? 1 : 0;
        if (tile == ntiles - 1 && !failed) plan->s = excl + total;
      }
    }
    __syncthreads();
    if (s_fail) break;
    const u32 excl = s_excl;
    #pragma unroll
    for (int r = 0; r < K2_PAIRS; ++r) {
      u32 pos = excl + s_wcnt[r * K2_WARPS + wid] + lane_pre[r];
      const u32 i0 = base + 2u * (r * K2_BLOCK + threadIdx.x);
      #pragma unroll
      for (int e = 0; e < 2; ++e) {
        if (keep[2 * r + e]) {
          if (pos < n) {
            keys_out[pos] = ((u64)(u32)(px[2 * r + e] - x0) << ybits) | (u64)(u32)(py[2 * r + e] - y0);
            idx_out[pos] = i0 + e;
          } else {
            flag_error(plan, ERR_INTERNAL);
          }
          ++pos;
        }
      }
    }
  }
  __syncthreads();
  for (u32 q = threadIdx.x; q < npasses * kRadix; q += K2_BLOCK) {
    u32 c = s_hist[q];
    if (c) atomicAdd(&(&plan->hist[0][0])[q], c);
  }
}

}  // namespace

int k2_tile() { return K2_TILE; }

cudaError_t k2_occupancy(int* blocks) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, k2_filter<true>, K2_BLOCK, 0);
}

cudaError_t launch_k2(const int* xy, Plan* plan, u64* keys_out, u32* idx_out, u64* status,
                      int grid, cudaStream_t st) {
  const bool vec = (reinterpret_cast<uintptr_t>(xy) & 15u) == 0;
  if (vec)
    k2_filter<true><<<grid, K2_BLOCK, 0, st>>>(xy, plan, keys_out, idx_out, status);
  else
    k2_filter<false><<<grid, K2_BLOCK, 0, st>>>(xy, plan, keys_out, idx_out, status);
  return cudaGetLastError();
}

}  // namespace gbh
