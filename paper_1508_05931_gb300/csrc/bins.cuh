// Bin starts and groups of the bucket sort (k3_bucket.cu), computed by one
// whole block from the bins' totals; shared by the bin scans (k3_bucket.cu)
// and the last block of the fused filter (k2_fused.cu), which supplies its
// own shared memory.
#pragma once

#include "hull_internal.cuh"

namespace gbh {

namespace {

constexpr int BS_BLOCK = 512;
constexpr int BS_WARPS = BS_BLOCK / 32;
constexpr int BS_PER = kBins / BS_BLOCK;    // bins per thread in the last block (a flag word each)
static_assert(BS_PER >= 1 && BS_PER <= 32 && BS_PER * BS_BLOCK == kBins, "whole slices of at most 32 bins per thread");

// Shared memory of bins_to_groups.
struct BinScanSmem {
  __align__(16) u32 v[kBins];       // totals, then starts (coalesced global access)
  u32 last_st[BS_BLOCK], last_cn[BS_BLOCK];
  u32 w[BS_WARPS];
};

// One whole block (BS_BLOCK threads): the bins' starts (bstart, and the
// split's cursors fcur when given) from their totals, the groups of
// consecutive bins, the survivor count.  Thread t owns bins
// [t BS_PER, t BS_PER + BS_PER).  `totals` may be bstart itself; VOL when
// other blocks of the same launch wrote it.
template <bool VOL>
__device__ void bins_to_groups(const u32* totals, Plan* plan, u32* __restrict__ bstart, uint2* __restrict__ groups,
                               u32* __restrict__ fcur, BinScanSmem& B) {
  u32* s_w = B.w;
  u32* s_last_st = B.last_st;
  u32* s_last_cn = B.last_cn;
  u32* s_v = B.v;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  static_assert(BS_PER % 4 == 0, "whole uint4 slices");
  {
    u32 v[BS_PER];
    #pragma unroll
    for (int j = 0; j < BS_PER; ++j) {
      const u32* p = &totals[threadIdx.x + j * BS_BLOCK];
      v[j] = VOL ? ld_volatile_u32(p) : *p;
    }
    #pragma unroll
    for (int j = 0; j < BS_PER; ++j) s_v[threadIdx.x + j * BS_BLOCK] = v[j];
  }
  __syncthreads();
  u32 cn[BS_PER], st[BS_PER];
  u32 tsum = 0;
  #pragma unroll
  for (int j = 0; j < BS_PER; j += 4) {
    const uint4 v = *reinterpret_cast<const uint4*>(&s_v[threadIdx.x * BS_PER + j]);
    cn[j] = v.x; cn[j + 1] = v.y; cn[j + 2] = v.z; cn[j + 3] = v.w;
  }
  #pragma unroll
  for (int j = 0; j < BS_PER; ++j) tsum += cn[j];
  u32 inc = tsum;
  #pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const u32 t = __shfl_up_sync(0xFFFFFFFFu, inc, o);
    if (lane >= o) inc += t;
  }
  if (lane == 31) s_w[wid] = inc;
  __syncthreads();
  u32 acc = inc - tsum;
  for (int w = 0; w < wid; ++w) acc += s_w[w];
  #pragma unroll
  for (int j = 0; j < BS_PER; ++j) { st[j] = acc; acc += cn[j]; }
  s_last_st[threadIdx.x] = st[BS_PER - 1];
  s_last_cn[threadIdx.x] = cn[BS_PER - 1];
  __syncthreads();
  const u32 T = (u32)kGroupTarget;
  u32 flags = 0;
  #pragma unroll
  for (int j = 0; j < BS_PER; ++j) {
    const u32 b = threadIdx.x * BS_PER + j;
    u32 pst, pcn;
    if (j) { pst = st[j - 1]; pcn = cn[j - 1]; }
    else if (threadIdx.x) { pst = s_last_st[threadIdx.x - 1]; pcn = s_last_cn[threadIdx.x - 1]; }
    else { pst = 0; pcn = 0; }
    const bool f = b % kFinePerCoarse == 0 || st[j] / T != pst / T || cn[j] > T || pcn > T;
    flags |= (u32)f << j;
  }
  const u32 nf = __popc(flags);
  u32 finc = nf;
  #pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const u32 t = __shfl_up_sync(0xFFFFFFFFu, finc, o);
    if (lane >= o) finc += t;
  }
  __syncthreads();
  if (lane == 31) s_w[wid] = finc;
  __syncthreads();
  u32 g = finc - nf;
  for (int w = 0; w < wid; ++w) g += s_w[w];
  #pragma unroll
  for (int j = 0; j < BS_PER; ++j) {
    if (flags & (1u << j)) groups[g++] = make_uint2(st[j], threadIdx.x * BS_PER + j);
  }
  #pragma unroll
  for (int j = 0; j < BS_PER; j += 4)
    *reinterpret_cast<uint4*>(&s_v[threadIdx.x * BS_PER + j]) = make_uint4(st[j], st[j + 1], st[j + 2], st[j + 3]);
  __syncthreads();
  for (u32 q = threadIdx.x; q < (u32)kBins; q += BS_BLOCK) {
    const u32 v = s_v[q];
    bstart[q] = v;
    if (fcur) fcur[q] = v;
  }
  if (threadIdx.x == BS_BLOCK - 1) {
    groups[g] = make_uint2(acc, (u32)kBins);
    plan->s = acc;            // the survivors: every bin's count
    plan->ngroups = g;
    plan->npasses = 0;        // no radix passes on this path;
    plan->sorted_in_b = 1;    // k3_bucket leaves the sorted survivors in the second buffer
  }
}
}  // namespace

}  // namespace gbh
