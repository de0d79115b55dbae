// Internal definitions shared by the sm_103a kernels of the hull pipeline.
//
// The pipeline follows Section 2.1 of Mei, "gScan: Accelerating Graham Scan
// on the GPU" (arXiv 1508.05931), steps 1-8, every step on the device:
//   K1 extremes (step 1)  ->  K2 quadrilateral filter + compaction (steps 2-3)
//   -> K3 onesweep radix sort (step 4)  ->  K4 region split + second-round
//   filter (steps 5-7, Figure 2 as an exclusive prefix-max scan)
//   -> K5 monotone-chain finalisation (step 8).
// A small device-resident Plan carries the sizes and parameters from one
// kernel to the next, so the host never synchronises inside a call.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

namespace gbh {

typedef unsigned long long u64;
typedef unsigned int u32;

constexpr int kCoordLimit = 1 << 29;     // |x|, |y| <= 2^29
constexpr int kMaxCorners = 12;          // filter polygon: 4 (quad) or up to 12 (learned)
constexpr int kRadixBits = 8;
constexpr int kRadix = 1 << kRadixBits;
constexpr int kMaxPasses = 8;            // 64-bit keys / 8-bit digits
constexpr u32 kMaxN = (1u << 30) - 1;    // look-back count fields are 30 bits

// Bucket sort of the survivors (the hull pipeline's sort): the first round
// scatters every survivor into one of kBins bins by the top kBinBits of its
// key; consecutive bins form groups of at most kGroupCap survivors, each
// sorted in shared memory by one block (sub-bins of the next kSubBits key
// bits, then the few keys of a sub-bin in place).
#ifndef GBH_GROUP_CAP
#define GBH_GROUP_CAP 8192
#endif
#ifndef GBH_SUB_BITS
#define GBH_SUB_BITS 12
#endif
constexpr int kBinBits = 13;
constexpr int kBins = 1 << kBinBits;
constexpr int kGroupCap = GBH_GROUP_CAP;     // survivors sorted in shared memory at once
constexpr int kGroupTarget = kGroupCap / 2;  // window of the group rule (see k3_bucket.cu)
constexpr int kSubBits = GBH_SUB_BITS;
// The filter's survivors are placed into kCoarse coarse bins (the top
// kCoarseBits of a bin); k3_split then spreads every coarse bin over its
// fine bins.
constexpr int kCoarseBits = 8;
constexpr int kCoarse = 1 << kCoarseBits;
constexpr int kFinePerCoarse = kBins / kCoarse;
constexpr int kBinPrefixBlocks = 64;           // most block totals k_bin_prefix keeps after the bins
constexpr int kSubBins = 1 << kSubBits;
// The fused front's witnesses come from every kSampleStride-th point, which
// K1 copies out while it reads them.
constexpr u32 kSampleStride = 32;
// Witness bins: the top kWitnessBits of the key (coarser than the sort's bins,
// so that the fused filter's table of witness directions, 2 x 8 bytes per
// bin, fits in shared memory beside its per-warp staging slices).
constexpr int kWitnessBits = 12;
constexpr int kWitnessBins = 1 << kWitnessBits;

// Error bits accumulated in Plan::error by the kernels.
enum : u32 {
  ERR_RANGE = 1u,       // a coordinate beyond +-2^29
  ERR_TIMEOUT = 2u,     // a bounded device wait ran out
  ERR_CAPACITY = 4u,    // output capacity below the hull size
  ERR_INTERNAL = 8u,    // an index left its buffer (skipped, never written)
  ERR_FALLBACK = 16u,   // a bin too large for the bucket sort: the call reruns on the radix passes
};

// Each call consumes kEpochStride epochs; look-back status words carry the
// epoch in their top 32 bits so stale words from earlier calls never match.
constexpr u32 kEpochStride = 16;
enum EpochSlot : u32 { EP_FILTER = 1, EP_SORT0 = 2, EP_REGION = 2 + kMaxPasses, EP_FINAL = 3 + kMaxPasses };

// Counters (dynamic tile ids, barriers), zeroed by K1 for every call.
enum CounterSlot : int {
  CTR_FILTER = 0,
  CTR_SORT0 = 1,                          // .. CTR_SORT0 + kMaxPasses - 1
  CTR_REGION = 1 + kMaxPasses,
  CTR_REGION2 = 2 + kMaxPasses,
  CTR_FINAL_BAR = 3 + kMaxPasses,
  CTR_FINAL_BAR_GEN = 4 + kMaxPasses,
  CTR_BIN_SCAN = 5 + kMaxPasses,          // last-block counter of the bin scan
  CTR_BIN_GROUP = 6 + kMaxPasses,         // next group of the bucket sort
  CTR_SPLIT = 7 + kMaxPasses,             // next tile of the coarse-to-fine split
  CTR_GROUP_AGG = 8 + kMaxPasses,         // last-block counter of the group aggregates
  CTR_WITNESS = 9 + kMaxPasses,           // last-block counter of the sampled witnesses
  CTR_FUSED = 10 + kMaxPasses,            // next output slot of the fused filter
  CTR_FUSED_DONE = 11 + kMaxPasses,       // last-block counter of the fused filter
  kNumCounters = 20,
};

struct ExtPartial {
  u64 key[4];
  u32 idx[4];
};

// The single-read front's sample polygon (k0_poly.cu builds it, K1 filters
// with it).  The first part is cleared before every call with the bins.
constexpr int kPolyDirs = 32;          // directions of the sample's extreme points
constexpr int kPolySlabs = 4096;       // most x slabs of the polygon's table
struct PolyTab {
  // cleared per call
  u64 best[kPolyDirs];   // per direction: (ordered projection << 32 | ~sample index), maximum
  u32 raw_count;         // K1's survivors: points on or outside the polygon
  u32 done;              // last-block counter of k0
  u32 pad[2];
  // written by k0's last block
  int ok;                // 1: at least 3 corners and an x range with an interior
  int k;                 // corners (counter-clockwise from the lexicographic minimum)
  int xl, xr;            // x of the leftmost and of the rightmost corner
  u32 sh;                // slab s holds x in [xl + s 2^sh, xl + (s + 1) 2^sh)
  u32 nslab;
  u32 pad2[2];
  int2 yb[kPolySlabs];    // per slab (ylo, yhi): a point of the slab with ylo < y < yhi is strictly
                         // inside (ylo >= the lower chain, yhi <= the upper chain over the slab)
};
constexpr size_t kPolyClearBytes = offsetof(PolyTab, ok);

struct Plan {
  // summary fields first: the host copies back everything before `ctr`
  u32 n;
  u32 spin_limit;
  u32 epoch;            // base epoch of the current call
  u32 error;
  u32 s;                // survivors of the first round (on the fused path: those left
                        // after the sampled-witness test, the sort's input)
  u32 s_quad;           // survivors of the first-round filter polygon alone
  u32 s_raw;            // single-read front: points on or outside the sample polygon
  u32 r_lo, r_up;       // survivors of the second round per region
  u32 h;                // hull size
  u32 h_lo, h_up;       // chain lengths (including both endpoints)
  int32_t ncorner;
  int32_t learned_used; // 1 when a learned polygon replaced the quad
  int32_t ext_idx[4];   // P_minx, P_maxx, P_miny, P_maxy
  int32_t ext_x[4], ext_y[4];
  int32_t cx[kMaxCorners], cy[kMaxCorners];
  int32_t key_x0, key_y0;   // key origin (bounding-box minimum)
  u32 ybits, kbits, npasses;
  u32 sorted_in_b;      // 1: the sorted survivors are in the second key/index buffer
  u32 fshift;           // bucket sort: bin = key >> fshift
  u32 ngroups;          // bucket sort: groups of consecutive bins
  u32 k1_done;          // last-block counter of K1 (self-resetting)
  // per-call scratch
  u32 ctr[kNumCounters];
  u32 hist[kMaxPasses][kRadix];   // digit histograms of the survivors' keys
};

// ---------------------------------------------------------------- helpers

__device__ __forceinline__ u64 ld_acquire_u64(const u64* p) {
  u64 v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_u64(u64* p, u64 v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
// Relaxed (gpu-scope) accesses for look-back words whose value is
// self-contained (flag and count in one 64-bit word): no fence is needed.
__device__ __forceinline__ u64 ld_relaxed_u64(const u64* p) {
  u64 v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed_u64(u64* p, u64 v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ u32 ld_volatile_u32(const u32* p) {
  return *reinterpret_cast<const volatile u32*>(p);
}
__device__ __forceinline__ void flag_error(Plan* plan, u32 bit) { atomicOr(&plan->error, bit); }
__device__ __forceinline__ bool aborted(const Plan* plan) {
  return (ld_volatile_u32(&plan->error) & (ERR_TIMEOUT | ERR_INTERNAL | ERR_FALLBACK)) != 0;
}

// Exact orientation (b - a) x (c - a) in int64.  Coordinates are bounded by
// 2^29, so each difference fits in int32 and each product in 2^60.
__device__ __forceinline__ long long orient(int ax, int ay, int bx, int by, int cx, int cy) {
  int ux = bx - ax, uy = by - ay, vx = cx - ax, vy = cy - ay;
  return (long long)ux * vy - (long long)uy * vx;
}
// Cross product of two direction vectors (differences of bounded points).
__device__ __forceinline__ long long cross2(int ax, int ay, int bx, int by) {
  return (long long)ax * by - (long long)ay * bx;
}

// Rounds a device-side wait (look-back, grid barrier) spins before it gives
// up with ERR_TIMEOUT, unless the caller's configuration sets another limit;
// every entry point that launches the pipeline uses it.
constexpr u32 kDefaultSpinLimit = 1u << 22;
// Look-back status word: [epoch:32 | flag:2 | count:30].
constexpr u32 ST_AGG = 1, ST_INCL = 2;
// ---- Bulk asynchronous copies (TMA, non-tensor) into shared memory.
// One thread arms an mbarrier with the expected byte count and issues a
// cp.async.bulk; consumers wait on the barrier's phase parity.  Source and
// destination must be 16-byte aligned and the size a multiple of 16.
constexpr u32 kBulkWaitLimit = 1u << 24;   // try_wait rounds before a wait gives up

__device__ __forceinline__ u32 smem_addr(const void* p) {
  return (u32)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(u64* bar, u32 count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
// Makes initialised barriers visible to the async proxy (then __syncthreads).
__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// Returns the barrier state token (unused by the callers: they wait on parity).
__device__ __forceinline__ u64 mbar_arrive_expect_tx(u64* bar, u32 bytes) {
  u64 state;
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 %0, [%1], %2;"
               : "=l"(state) : "r"(smem_addr(bar)), "r"(bytes) : "memory");
  return state;
}
__device__ __forceinline__ void bulk_load(void* dst, const void* src, u32 bytes, u64* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
      ::"r"(smem_addr(dst)), "l"(src), "r"(bytes), "r"(smem_addr(bar)) : "memory");
}
// L2 eviction policies (createpolicy) for streaming reads that nothing
// reads again (evict_first) and for scattered writes that should stay in L2
// until their sectors are complete (evict_last).
__device__ __forceinline__ u64 policy_evict_first() {
  u64 p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ u64 policy_evict_last() {
  u64 p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ void bulk_load_hint(void* dst, const void* src, u32 bytes, u64* bar, u64 pol) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;"
      ::"r"(smem_addr(dst)), "l"(src), "r"(bytes), "r"(smem_addr(bar)), "l"(pol) : "memory");
}
// Asynchronous global -> shared copies (no registers held while in flight).
__device__ __forceinline__ void cp_async4(void* smem_dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_addr(smem_dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async8(void* smem_dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_addr(smem_dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async16(void* smem_dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(smem_dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Bulk prefetch into L2 of elements [lo, hi) of an array of `esz`-byte
// elements, widened to 16-byte boundaries (the allocation must extend 16
// bytes past element hi) and cut to `cap` bytes.
__device__ __forceinline__ void prefetch_span_l2(const void* base, u32 lo, u32 hi, u32 esz, u32 cap) {
  if (hi <= lo) return;
  const uintptr_t a = (reinterpret_cast<uintptr_t>(base) + (uintptr_t)lo * esz) & ~(uintptr_t)15;
  const uintptr_t b = (reinterpret_cast<uintptr_t>(base) + (uintptr_t)hi * esz + 15) & ~(uintptr_t)15;
  const u32 bytes = (u32)min((uintptr_t)cap, b - a) & ~15u;
  if (bytes) asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a), "r"(bytes) : "memory");
}

// Read-only loads with an L2 eviction policy.
__device__ __forceinline__ u64 ld_hint_u64(const u64* p, u64 pol) {
  u64 v;
  asm("ld.global.nc.L2::cache_hint.b64 %0, [%1], %2;" : "=l"(v) : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ u32 ld_hint_u32(const u32* p, u64 pol) {
  u32 v;
  asm("ld.global.nc.L2::cache_hint.b32 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ void st_hint_u64(u64* p, u64 v, u64 pol) {
  asm volatile("st.global.L2::cache_hint.b64 [%0], %1, %2;" ::"l"(p), "l"(v), "l"(pol) : "memory");
}
__device__ __forceinline__ void st_hint_u32(u32* p, u32 v, u64 pol) {
  asm volatile("st.global.L2::cache_hint.b32 [%0], %1, %2;" ::"l"(p), "r"(v), "l"(pol) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(u64* bar, u32 parity) {
  u32 ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok) : "r"(smem_addr(bar)), "r"(parity) : "memory");
  return ok != 0u;
}
// Waits for the given phase of `bar` to complete; false if it did not within
// `limit` rounds (the call's spin limit for the waits of a ring; the fixed
// kBulkWaitLimit for the drain at a kernel's end).
__device__ __forceinline__ bool mbar_wait(u64* bar, u32 parity, u32 limit = kBulkWaitLimit) {
  for (u32 it = 0; it < limit; ++it)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

// Mask of the lanes whose 8-bit radix digit equals this lane's (all 32
// lanes take part): eight ballots, each compared with this lane's own bit
// made into a full mask.  Digit bits 7..4 become the byte sign bits of hi,
// bits 3..0 those of lo (the shifted copies do not overlap, so the products
// are plain ORs), and prmt with the sign flag in its selector replicates a
// byte's sign bit over the whole word.
__device__ __forceinline__ u32 warp_digit_peers(u32 dg) {
  static_assert(kRadixBits == 8, "two words of four byte sign bits");
  const u32 hi = dg * 0x08040201u;
  const u32 lo = (dg << 4) * 0x08040201u;
  u32 differ = 0u;
  #pragma unroll
  for (int b = 0; b < kRadixBits; ++b) {
    const u32 sel = 0x8888u + 0x1111u * (u32)(b & 3);
    u32 mine;
    asm("prmt.b32 %0, %1, 0, %2;" : "=r"(mine) : "r"(b < 4 ? hi : lo), "r"(sel));
    differ |= __ballot_sync(0xFFFFFFFFu, mine != 0u) ^ mine;
  }
  return ~differ;
}

__device__ __forceinline__ u64 make_status(u32 epoch, u32 flag, u32 count) {
  return ((u64)epoch << 32) | ((u64)flag << 30) | (u64)(count & 0x3FFFFFFFu);
}
__device__ __forceinline__ u32 status_flag(u64 w, u32 epoch) {
  return ((u32)(w >> 32) == epoch) ? (u32)((w >> 30) & 3u) : 0u;
}
__device__ __forceinline__ u32 status_count(u64 w) { return (u32)(w & 0x3FFFFFFFu); }

// Back-off used inside bounded waits.
__device__ __forceinline__ void spin_pause(u32 it) {
  if (it > 64) __nanosleep(it > 4096 ? 256 : 32);
}

// Warp-cooperative decoupled look-back over a single count (K2).  Lane l
// inspects tile (tile - 1 - l - 32*w) for windows w = 0, 1, ...; returns
// the exclusive prefix of this tile, identical on all lanes.  On a timeout
// (or another block's abort) sets ERR_TIMEOUT and returns 0.
__device__ __forceinline__ u32 warp_lookback_count(u64* status, u32 tile, u32 epoch,
                                                   Plan* plan, u32 spin_limit, bool* failed) {
  const int lane = threadIdx.x & 31;
  u32 excl = 0;
  long long base = (long long)tile - 1;
  *failed = false;
  while (base >= 0) {
    long long t = base - lane;
    u64 w = 0;
    u32 f = ST_INCL;   // lanes past tile 0 act as an empty inclusive prefix
    if (t >= 0) {
      u32 it = 0;
      for (;;) {
        w = ld_relaxed_u64(&status[t]);
        f = status_flag(w, epoch);
        if (f != 0) break;
        if (++it > spin_limit || aborted(plan)) { f = 0xFFu; break; }
        spin_pause(it);
      }
    }
    if (__any_sync(0xFFFFFFFFu, f == 0xFFu)) {
      if (lane == 0) flag_error(plan, ERR_TIMEOUT);
      *failed = true;
      return 0;
    }
    u32 incl_mask = __ballot_sync(0xFFFFFFFFu, f == ST_INCL);
    int stop = incl_mask ? (__ffs(incl_mask) - 1) : 31;   // nearest inclusive prefix
    u32 c = (t >= 0 && lane <= stop) ? status_count(w) : 0u;
    #pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xFFFFFFFFu, c, o);
    excl += c;
    if (incl_mask) break;
    base -= 32;
  }
  return excl;
}

// Block-wide decoupled look-back over a single count: thread i inspects
// tile (tile - 1 - i - blockDim.x * w) in window w, so a round trip covers
// blockDim.x predecessors.  Every thread of the block must call it; all get
// the same exclusive prefix.  On a timeout (or another block's abort) sets
// ERR_TIMEOUT and *failed.  `red` is shared scratch of >= blockDim.x / 32 + 2 words.
__device__ __forceinline__ u32 block_lookback_count(const u64* status, u32 tile, u32 epoch,
                                                    Plan* plan, u32 spin_limit, bool* failed,
                                                    u32* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nw = blockDim.x >> 5;
  u32 excl = 0;
  long long base = (long long)tile - 1;
  *failed = false;
  while (base >= 0) {
    const long long t = base - (long long)threadIdx.x;
    u64 w = 0;
    u32 f = 0;
    bool bad = false;
    if (t >= 0) {
      u32 it = 0;
      for (;;) {
        w = ld_relaxed_u64(&status[t]);
        f = status_flag(w, epoch);
        if (f != 0) break;
        if (++it > spin_limit || aborted(plan)) { bad = true; flag_error(plan, ERR_TIMEOUT); break; }
        spin_pause(it);
      }
    }
    // Nearest inclusive prefix: the lowest thread holding one.
    const u32 incl = __ballot_sync(0xFFFFFFFFu, t >= 0 && f == ST_INCL);
    if (threadIdx.x == 0) { red[nw] = 0xFFFFFFFFu; red[nw + 1] = 0u; }
    __syncthreads();
    if (lane == 0 && incl) atomicMin(&red[nw], (u32)(wid * 32 + __ffs(incl) - 1));
    if (bad) red[nw + 1] = 1u;
    __syncthreads();
    const u32 stop = red[nw];
    if (red[nw + 1]) {
      if (threadIdx.x == 0) flag_error(plan, ERR_TIMEOUT);
      *failed = true;
      __syncthreads();
      return 0;
    }
    u32 c = (t >= 0 && (u32)threadIdx.x <= stop) ? status_count(w) : 0u;
    #pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xFFFFFFFFu, c, o);
    __syncthreads();
    if (lane == 0) red[wid] = c;
    __syncthreads();
    u32 sum = 0;
    for (int q = 0; q < nw; ++q) sum += red[q];
    excl += sum;
    __syncthreads();
    if (stop != 0xFFFFFFFFu) break;
    base -= blockDim.x;
  }
  return excl;
}

}  // namespace gbh
