// K3: stable LSD radix sort of the survivors' (key, idx) pairs (Section 2.1
// step 4, Section 3.3), one onesweep pass per 8-bit digit.
//
// The digit histograms of all passes were accumulated by K2, so every pass
// is a single kernel: a block takes the next tile (dynamic id), ranks its
// keys by digit with warp match/popc (stable: items are ranked in input
// order), publishes its per-digit counts, resolves its global per-digit
// offsets by a decoupled look-back (one thread per digit, bounded waits),
// stages the tile in shared memory in digit order and writes it out, so
// that consecutive threads write consecutive addresses within each digit.
// Only the passes that the survivors' varying key bits need are run; the
// others return at once, and the Plan records where the result ends up.
#include "hull_internal.cuh"
#include "kernels.h"

namespace gbh {

namespace {

constexpr int K3_BLOCK = 256;
constexpr int K3_WARPS = K3_BLOCK / 32;
constexpr int K3_ITEMS = 16;
constexpr int K3_TILE = K3_BLOCK * K3_ITEMS;      // 4096 keys
constexpr int K3_WARP_ITEMS = 32 * K3_ITEMS;      // 512 keys per warp
static_assert(K3_BLOCK == kRadix, "one thread per digit");

__global__ void __launch_bounds__(K3_BLOCK, 3)
k3_onesweep(const u64* __restrict__ keys_in, const u32* __restrict__ idx_in,
            u64* __restrict__ keys_out, u32* __restrict__ idx_out, Plan* plan,
            u64* __restrict__ status, u32 pass) {
  extern __shared__ __align__(16) unsigned char k3_smem[];
  u64* s_keys = reinterpret_cast<u64*>(k3_smem);
  u32* s_idx = reinterpret_cast<u32*>(k3_smem + K3_TILE * sizeof(u64));
  __shared__ unsigned short s_whist[K3_WARPS][kRadix];
  __shared__ u32 s_gstart[kRadix];
  __shared__ u32 s_tstart[kRadix];
  __shared__ u32 s_gbase[kRadix];
  __shared__ u32 s_warp_tot[K3_WARPS];
  __shared__ u32 s_tile;
  __shared__ int s_fail;

  if (pass >= plan->npasses || (plan->error & ERR_RANGE)) return;
  const u32 s = plan->s;
  const u32 shift = pass * kRadixBits;
  const u32 epoch = plan->epoch + EP_SORT0 + pass;
  const u32 spin = plan->spin_limit;
  const u32 ntiles = (s + K3_TILE - 1) / K3_TILE;
  const int d = threadIdx.x;      // this thread's digit in the per-digit phases
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const u32 lt_mask = (1u << lane) - 1u;

  // Global exclusive start of every digit (block scan of the histogram).
  {
    u32 v = plan->hist[pass][d];
    u32 inc = v;
    #pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      u32 t = __shfl_up_sync(0xFFFFFFFFu, inc, o);
      if (lane >= o) inc += t;
    }
    if (lane == 31) s_warp_tot[wid] = inc;
    __syncthreads();
    u32 off = 0;
    for (int w = 0; w < wid; ++w) off += s_warp_tot[w];
    s_gstart[d] = off + inc - v;
  }

  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) s_tile = atomicAdd(&plan->ctr[CTR_SORT0 + pass], 1u);
    for (int w = 0; w < K3_WARPS; ++w) s_whist[w][d] = 0;
    __syncthreads();
    const u32 tile = s_tile;
    if (tile >= ntiles) break;
    const u32 base = tile * (u32)K3_TILE;
    const u32 tile_n = min((u32)K3_TILE, s - base);

    u64 key[K3_ITEMS];
    u32 idx[K3_ITEMS];
    unsigned short rank[K3_ITEMS];
    const u32 wbase = base + wid * K3_WARP_ITEMS;
    #pragma unroll
    for (int it = 0; it < K3_ITEMS; ++it) {
      u32 p = wbase + it * 32 + lane;
      if (p < s) { key[it] = keys_in[p]; idx[it] = idx_in[p]; }
      else { key[it] = 0; idx[it] = 0; }
    }
    // Stable in-warp ranking, item by item in input order.
    #pragma unroll
    for (int it = 0; it < K3_ITEMS; ++it) {
      const bool valid = (wbase + it * 32 + lane) < s;
      const u32 vmask = __ballot_sync(0xFFFFFFFFu, valid);
      const u32 dg = (u32)(key[it] >> shift) & (kRadix - 1);
      u32 peers = 0, before = 0;
      if (valid) {
        peers = __match_any_sync(vmask, dg);
        before = s_whist[wid][dg];
      }
      __syncwarp();
      if (valid) {
        rank[it] = (unsigned short)(before + __popc(peers & lt_mask));
        if (lane == 31 - __clz(peers)) s_whist[wid][dg] = (unsigned short)(before + __popc(peers));
      }
      __syncwarp();
    }
    __syncthreads();

    // Per digit: warp offsets, tile count, publish, look-back.
    u32 cnt = 0;
    #pragma unroll
    for (int w = 0; w < K3_WARPS; ++w) {
      u32 c = s_whist[w][d];
      s_whist[w][d] = (unsigned short)cnt;
      cnt += c;
    }
    u64* st = status + (size_t)tile * kRadix + d;
    if (tile == 0) st_release_u64(st, make_status(epoch, ST_INCL, cnt));
    else st_release_u64(st, make_status(epoch, ST_AGG, cnt));
    // Tile-local exclusive digit starts (block scan of cnt).
    {
      u32 inc = cnt;
      #pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        u32 t = __shfl_up_sync(0xFFFFFFFFu, inc, o);
        if (lane >= o) inc += t;
      }
      if (lane == 31) s_warp_tot[wid] = inc;
      __syncthreads();
      u32 off = 0;
      for (int w = 0; w < wid; ++w) off += s_warp_tot[w];
      s_tstart[d] = off + inc - cnt;
    }
    u32 excl = 0;
    bool fail = false;
    if (tile > 0) {
      long long t = (long long)tile - 1;
      while (t >= 0) {
        const u64* sp = status + (size_t)t * kRadix + d;
        u64 w;
        u32 f;
        u32 it = 0;
        for (;;) {
          w = ld_acquire_u64(sp);
          f = status_flag(w, epoch);
          if (f != 0) break;
          if (++it > spin || aborted(plan)) { fail = true; break; }
          spin_pause(it);
        }
        if (fail) break;
        excl += status_count(w);
        if (f == ST_INCL) break;
        --t;
      }
      if (!fail) st_release_u64(st, make_status(epoch, ST_INCL, excl + cnt));
    }
    if (fail) flag_error(plan, ERR_TIMEOUT);
    s_gbase[d] = s_gstart[d] + excl - s_tstart[d];
    if (threadIdx.x == 0) s_fail = 0;
    __syncthreads();
    if (fail) s_fail = 1;
    __syncthreads();
    if (s_fail) break;

    // Stage the tile in digit order, then write it out.
    #pragma unroll
    for (int it = 0; it < K3_ITEMS; ++it) {
      if (wbase + it * 32 + lane < s) {
        const u32 dg = (u32)(key[it] >> shift) & (kRadix - 1);
        const u32 lp = s_tstart[dg] + s_whist[wid][dg] + rank[it];
        s_keys[lp] = key[it];
        s_idx[lp] = idx[it];
      }
    }
    __syncthreads();
    for (u32 j = threadIdx.x; j < tile_n; j += K3_BLOCK) {
      const u64 k = s_keys[j];
      const u32 dg = (u32)(k >> shift) & (kRadix - 1);
      const u32 gp = s_gbase[dg] + j;
      if (gp < s) {
        keys_out[gp] = k;
        idx_out[gp] = s_idx[j];
      } else {
        flag_error(plan, ERR_INTERNAL);
      }
    }
  }
}

}  // namespace

int k3_tile() { return K3_TILE; }
size_t k3_dyn_smem() { return (size_t)K3_TILE * (sizeof(u64) + sizeof(u32)); }

cudaError_t k3_configure() {
  return cudaFuncSetAttribute(k3_onesweep, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)k3_dyn_smem());
}

cudaError_t k3_occupancy(int* blocks) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, k3_onesweep, K3_BLOCK, k3_dyn_smem());
}

cudaError_t launch_k3(const u64* kin, const u32* iin, u64* kout, u32* iout, Plan* plan,
                      u64* status, u32 pass, int grid, cudaStream_t st) {
  k3_onesweep<<<grid, K3_BLOCK, k3_dyn_smem(), st>>>(kin, iin, kout, iout, plan, status, pass);
  return cudaGetLastError();
}

}  // namespace gbh
