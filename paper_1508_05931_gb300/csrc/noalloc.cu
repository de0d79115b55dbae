// hull_compute_noalloc: the hull pipeline with every piece of scratch memory
// taken from one file-scope device array instead of a context workspace.
//
// Who needs it: callers that must not allocate device memory at all --
// code running where a cudaMalloc is forbidden or unsafe (inside a host
// callback or a memory-pool hook, in a plug-in whose host application owns
// the whole device memory budget), and latency-critical callers that cannot
// afford the implicit device synchronisation that cudaMalloc/cudaFree may
// perform.  They pass their own input and output buffers; everything else
// lives in g_noalloc_scratch below.
//
// Limits and sharing rules (also stated in include/gbhull.h):
//   - at most HULL_NOALLOC_MAX_POINTS points per call;
//   - g_noalloc_scratch (HULL_NOALLOC_SCRATCH_BYTES) exists on every GPU on
//     which this library is loaded, for the life of the process;
//   - every call on a device uses the same array and leaves its contents
//     behind; the parts that must start at zero (the Plan and the look-back
//     status words) are cleared at the start of every call;
//   - calls that overlap on the GPU (different streams, or different host
//     threads on one device) race on the array: serialise them;
//   - the first call on each device performs a one-time set-up (symbol
//     address lookup, kernel attributes, occupancy queries) with that device
//     current; make that first call before any stream capture.
#include <cstddef>
#include <cstdint>
#include <mutex>

#include "../../include/gbhull.h"
#include "hull_internal.cuh"
#include "kernels.h"

using namespace gbh;

namespace {

constexpr size_t kNoAllocBytes = HULL_NOALLOC_SCRATCH_BYTES;
constexpr int kMaxDevices = 64;

// The scratch array.  Host code must not use this name as an address: it
// is resolved per device with cudaGetSymbolAddress in noalloc_setup().
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

struct NoAllocDevice {
  bool ready = false;
  unsigned char* base = nullptr;   // device address of g_noalloc_scratch
  int num_sms = 0;
  int occ_k2c = 1, occ_k2 = 1, occ_k3 = 1, occ_k4 = 1, occ_k5 = 1;
};

NoAllocDevice g_dev[kMaxDevices];
std::mutex g_setup_mutex;

size_t up256(size_t v) { return (v + 255) & ~size_t(255); }

struct Carve {
  Plan* plan;
  u64* st_filter;
  u64* st_sort;
  void* st_region;
  size_t zero_bytes;   // plan + status words, cleared on every call
  ExtPartial* partials;
  u64* keys[2];
  u32* idx[2];
  int2* lo_xy; int* lo_idx; int2* up_xy; int* up_idx;
  int2* h_xy[2]; int* h_idx[2];
  u32* cnt[2];
  int4* jobs;
  unsigned char* mask;
  size_t total;
};

// Lays the pipeline's buffers for HULL_NOALLOC_MAX_POINTS points out in the
// array; with base == nullptr it only measures.
Carve carve(unsigned char* base, int num_sms) {
  const size_t cap = HULL_NOALLOC_MAX_POINTS;
  const size_t chunk = (size_t)k5_chunk();
  const size_t t2 = (cap + k2_tile() - 1) / k2_tile() + 1;
  const size_t t3 = (cap + k3_tile() - 1) / k3_tile() + 1;
  const size_t t4 = (cap + k4_tile() - 1) / k4_tile() + 1;
  const size_t slots = cap + 4 + 2 * chunk;
  const size_t nchunks = slots / (size_t)k5_min_chunk() + 2;
  const size_t parts = (size_t)num_sms * 4 + 8;
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t o = off; off = up256(off + bytes); return base + o; };
  Carve c{};
  c.plan = reinterpret_cast<Plan*>(take(sizeof(Plan)));
  c.st_filter = reinterpret_cast<u64*>(take(t2 * 8));
  c.st_sort = reinterpret_cast<u64*>(take(t3 * kRadix * 8));
  c.st_region = take(t4 * k4_status_bytes());
  c.zero_bytes = off;
  c.partials = reinterpret_cast<ExtPartial*>(take(parts * sizeof(ExtPartial)));
  for (int b = 0; b < 2; ++b) c.keys[b] = reinterpret_cast<u64*>(take(cap * 8));
  for (int b = 0; b < 2; ++b) c.idx[b] = reinterpret_cast<u32*>(take(cap * 4));
  c.lo_xy = reinterpret_cast<int2*>(take((cap + 2) * 8));
  c.lo_idx = reinterpret_cast<int*>(take((cap + 2) * 4));
  c.up_xy = reinterpret_cast<int2*>(take((cap + 2) * 8));
  c.up_idx = reinterpret_cast<int*>(take((cap + 2) * 4));
  for (int b = 0; b < 2; ++b) {
    c.h_xy[b] = reinterpret_cast<int2*>(take(slots * 8));
    c.h_idx[b] = reinterpret_cast<int*>(take(slots * 4));
  }
  for (int b = 0; b < 2; ++b) c.cnt[b] = reinterpret_cast<u32*>(take(nchunks * 4));
  c.jobs = reinterpret_cast<int4*>(take(nchunks * 16));
  c.mask = take(cap / 8 + 4096);
  c.total = off;
  return c;
}

int grid_for(int occ, int num_sms, size_t work) {
  size_t g = (size_t)occ * (size_t)num_sms;
  if (work < g) g = work;
  return g < 1 ? 1 : (int)g;
}

// One-time set-up for the current device (called with it current).
hull_status noalloc_setup(int dev, NoAllocDevice** out) {
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  NoAllocDevice& d = g_dev[dev];
  if (!d.ready) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      return HULL_ECUDA;
    }
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) { cudaGetLastError(); return HULL_ECUDA; }
    if (carve(nullptr, prop.multiProcessorCount).total > kNoAllocBytes) return HULL_EINTERNAL;
    if (k2_configure() != cudaSuccess || k3_configure() != cudaSuccess ||
        k5_configure(&d.occ_k5) != cudaSuccess ||
        k2_occupancy(&d.occ_k2c, &d.occ_k2) != cudaSuccess || k3_occupancy(&d.occ_k3) != cudaSuccess ||
        k4_occupancy(&d.occ_k4) != cudaSuccess || d.occ_k5 < 1) {
      cudaGetLastError();
      return HULL_ECUDA;
    }
    d.base = static_cast<unsigned char*>(p);
    d.num_sms = prop.multiProcessorCount;
    d.ready = true;
  }
  *out = &d;
  return HULL_OK;
}

}  // namespace

extern "C" hull_status hull_compute_noalloc(const int32_t* d_xy, int64_t n, int32_t* d_out,
                                            int64_t cap, int64_t* h_count, void* stream) {
  if (!h_count || n < 0 || cap < 0) return HULL_EINVAL;
  if (n > (int64_t)HULL_NOALLOC_MAX_POINTS) return HULL_EINVAL;
  if (n > 0 && (!d_xy || (reinterpret_cast<uintptr_t>(d_xy) & 7u) != 0)) return HULL_EINVAL;
  if (cap > 0 && !d_out) return HULL_EINVAL;
  *h_count = 0;
  if (n == 0) return HULL_OK;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return HULL_ECUDA;
  }
  NoAllocDevice* d = nullptr;
  hull_status r = noalloc_setup(dev, &d);
  if (r != HULL_OK) return r;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Carve c = carve(d->base, d->num_sms);
  const u32 un = (u32)n;

  cudaError_t e = cudaMemsetAsync(c.plan, 0, c.zero_bytes, st);
  if (e == cudaSuccess)
    e = launch_k1(d_xy, un, kDefaultSpinLimit, c.plan, c.partials, k1_grid(un, d->num_sms), st);
  const size_t t2 = (un + k2_tile() - 1) / k2_tile();
  if (e == cudaSuccess)
    e = launch_k2(d_xy, c.plan, c.keys[0], c.idx[0], c.st_filter, c.mask, grid_for(d->occ_k2c, d->num_sms, t2),
                   grid_for(d->occ_k2, d->num_sms, t2), st);
  const size_t t3 = (un + k3_tile() - 1) / k3_tile();
  for (u32 p = 0; p < (u32)kMaxPasses && e == cudaSuccess; ++p)
    e = launch_k3(c.keys[p & 1], c.idx[p & 1], c.keys[(p + 1) & 1], c.idx[(p + 1) & 1], c.plan,
                  c.st_sort, p, grid_for(d->occ_k3, d->num_sms, t3), st);
  const size_t t4 = (un + k4_tile() - 1) / k4_tile();
  if (e == cudaSuccess)
    e = launch_k4(c.keys[0], c.idx[0], c.keys[1], c.idx[1], c.plan, c.st_region, t4, c.lo_xy, c.lo_idx,
                  c.up_xy, c.up_idx, c.h_xy[0], c.h_idx[0], c.h_xy[1], c.h_idx[1],
                  grid_for(d->occ_k4, d->num_sms, t4), st);
  const size_t chunks = (un + 4) / (size_t)k5_chunk() + 2;
  if (e == cudaSuccess)
    e = launch_k5(c.lo_xy, c.lo_idx, c.up_xy, c.up_idx, c.plan, c.h_xy[0], c.h_idx[0], c.h_xy[1],
                  c.h_idx[1], c.cnt[0], c.cnt[1], c.jobs, d_out, (long long)cap,
                  grid_for(d->occ_k5 < 4 ? d->occ_k5 : 4, d->num_sms, chunks < 64 ? 64 : chunks), st);
  // Read the summary back into host stack memory (a pageable copy: no
  // pinned buffer is allocated) and wait for the stream.
  alignas(16) unsigned char summary[offsetof(Plan, ctr)];
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(summary, c.plan, sizeof(summary), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return HULL_ECUDA;
  }
  const Plan* p = reinterpret_cast<const Plan*>(summary);
  if (p->error & ERR_RANGE) return HULL_ERANGE;
  if (p->error & ERR_TIMEOUT) return HULL_ETIMEOUT;
  if (p->error & ERR_INTERNAL) return HULL_EINTERNAL;
  *h_count = p->h;
  if (p->error & ERR_CAPACITY) return HULL_ECAPACITY;
  return HULL_OK;
}
