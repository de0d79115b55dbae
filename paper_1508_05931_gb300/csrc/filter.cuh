// The first-round filter's per-point test (Section 2.1 step 2, Section
// 3.1), shared by the kernels that stream the points (k2_filter.cu,
// k2_fused.cu): the filter polygon's edges as multiply-add coefficients, the
// strict-interior test, and the chunked loads of the points (128-bit loads,
// or a ring of bulk copies into shared memory).
#pragma once

#include "hull_internal.cuh"

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

// Strict-interior test with the corner count known only at run time.
__device__ __forceinline__ bool strictly_inside_rt(const Edges& E, int k, int x, int y) {
  bool in = k >= 3;
  #pragma unroll
  for (int j = 0; j < kMaxCorners; ++j) {
    if (j < k) {
      const long long o = (long long)E.ex[j] * y + (long long)E.ney[j] * x + E.nc[j];
      in = in && (o > 0);
    }
  }
  return in;
}

}  // namespace

}  // namespace gbh
