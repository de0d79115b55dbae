// Small helper kernels: Plan set-up for the stage entry points, a
// stand-alone first-digit histogram (for sorting arbitrary keys), index
// fills and label gathers.
#include "hull_internal.cuh"
#include "kernels.h"

namespace gbh {

namespace {

__global__ void k_plan_patch(Plan* plan, PlanPatch p) {
  for (int q = threadIdx.x; q < kMaxPasses * kRadix; q += blockDim.x)
    if (p.zero_hist) (&plan->hist[0][0])[q] = 0u;
  for (int q = threadIdx.x; q < kNumCounters; q += blockDim.x)
    if (p.zero_counters) plan->ctr[q] = 0u;
  if (threadIdx.x != 0) return;
  if (p.new_call) {
    plan->epoch += kEpochStride;
    plan->error = 0u;
    plan->spin_limit = p.spin_limit;
  }
  if (p.set_s) plan->s = p.s;
  if (p.set_npasses) { plan->npasses = p.npasses; plan->sorted_in_b = p.npasses & 1u; }
  if (p.set_ncorner) plan->ncorner = p.ncorner;
  if (p.set_r) { plan->r_lo = p.r_lo; plan->r_up = p.r_up; }
}

// Histogram of the first radix digit (each radix pass counts the next one).
__global__ void k_hist(const u64* __restrict__ keys, Plan* plan) {
  __shared__ u32 h[kRadix];
  const u32 s = plan->s;
  for (int q = threadIdx.x; q < kRadix; q += blockDim.x) h[q] = 0u;
  __syncthreads();
  for (u32 i = blockIdx.x * blockDim.x + threadIdx.x; i < s; i += gridDim.x * blockDim.x)
    atomicAdd(&h[(u32)keys[i] & (kRadix - 1)], 1u);
  __syncthreads();
  for (u32 q = threadIdx.x; q < kRadix; q += blockDim.x)
    if (h[q]) atomicAdd(&plan->hist[0][q], h[q]);
}

__global__ void k_iota(int* out, u32 m) {
  for (u32 i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) out[i] = (int)i;
}

// out[i] = labels[pos[i]] for i < count (count read from the device).
__global__ void k_gather_labels(const int* __restrict__ pos, const int* __restrict__ labels,
                                const u32* count, u32 skip_first, int* __restrict__ out, u32 cap) {
  const u32 c = *count;
  for (u32 i = blockIdx.x * blockDim.x + threadIdx.x; i < c && i < cap; i += gridDim.x * blockDim.x)
    out[i] = labels[pos[i + skip_first]];
}

}  // namespace

cudaError_t launch_plan_patch(Plan* plan, const PlanPatch& p, cudaStream_t st) {
  k_plan_patch<<<1, 256, 0, st>>>(plan, p);
  return cudaGetLastError();
}

cudaError_t launch_hist(const u64* keys, Plan* plan, int grid, cudaStream_t st) {
  k_hist<<<grid, 512, 0, st>>>(keys, plan);
  return cudaGetLastError();
}

cudaError_t launch_iota(int* out, u32 m, cudaStream_t st) {
  int grid = (int)((m + 255) / 256);
  if (grid > 4096) grid = 4096;
  if (grid < 1) grid = 1;
  k_iota<<<grid, 256, 0, st>>>(out, m);
  return cudaGetLastError();
}

// The sorted survivors of the radix path as points: out_xy[i] = xy[idx[i]]
// and out_idx[i] = idx[i] for i < plan->s, idx being the index buffer that
// holds the sorted result (plan->sorted_in_b selects ib over ia).
__global__ void k_gather_sorted(const int2* __restrict__ xy, const u32* ia, const u32* ib, const Plan* plan,
                                int2* __restrict__ out_xy, int* __restrict__ out_idx, u32 cap) {
  const u32 s = plan->s;
  const u32* idx = plan->sorted_in_b ? ib : ia;
  for (u32 i = blockIdx.x * blockDim.x + threadIdx.x; i < s && i < cap; i += gridDim.x * blockDim.x) {
    const u32 j = idx[i];
    out_xy[i] = xy[j];
    out_idx[i] = (int)j;
  }
}

cudaError_t launch_gather_sorted(const int2* xy, const u32* ia, const u32* ib, const Plan* plan, int2* out_xy,
                                 int* out_idx, u32 cap, cudaStream_t st) {
  int grid = (int)((cap + 255) / 256);
  if (grid > 4096) grid = 4096;
  if (grid < 1) grid = 1;
  k_gather_sorted<<<grid, 256, 0, st>>>(xy, ia, ib, plan, out_xy, out_idx, cap);
  return cudaGetLastError();
}

cudaError_t launch_gather_labels(const int* pos, const int* labels, const u32* count,
                                 u32 skip_first, int* out, u32 cap, cudaStream_t st) {
  int grid = (int)((cap + 255) / 256);
  if (grid > 4096) grid = 4096;
  if (grid < 1) grid = 1;
  k_gather_labels<<<grid, 256, 0, st>>>(pos, labels, count, skip_first, out, cap);
  return cudaGetLastError();
}

}  // namespace gbh
