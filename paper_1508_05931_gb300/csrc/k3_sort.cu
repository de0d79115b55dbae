// K3: stable LSD radix sort of the survivors' (key, idx) pairs (Section 2.1
// step 4, Section 3.3), one onesweep pass per 8-bit digit.
//
// Each pass is one kernel.  A block takes the next tile (dynamic tile id,
// claimed when the block is ready to start it), counts the tile's digits per warp
// with shared-memory atomics and publishes the tile's counts at once, so
// that later tiles' look-backs find them early.  From the per-warp counts
// every warp knows its first position per digit, so ranking (stable: items
// in input order; lanes with equal digits found with ballots, the group's
// positions reserved by one atomic of its highest lane) writes each key
// straight to its place in a digit-ordered staging area in shared memory.
// A decoupled look-back (one thread per digit, K3_WINDOW status words in
// flight per step, bounded waits) gives the tile's global digit offsets,
// and the staged tile is written out with consecutive threads on
// consecutive addresses within each digit.  While it reads the keys a pass also counts the next
// digit, so pass p + 1 starts with its histogram complete (K2 counts the
// first digit).  Only the passes that the keys' varying bits need do work;
// the others return at once, and the Plan records where the result is.
#include "hull_internal.cuh"
#include "kernels.h"

namespace gbh {

namespace {

// Tuning knobs (tile shape and ranking primitive).
#ifndef K3_ITEMS_CFG
#define K3_ITEMS_CFG 16
#endif
#ifndef K3_MINBLOCKS_CFG
#define K3_MINBLOCKS_CFG 3
#endif
#ifndef K3_RANK_BALLOT
#define K3_RANK_BALLOT 3      // lanes with equal digits, from 8 ballots compared with this lane's
                              // bits as full masks made by prmt (3) or shifts (2), or with
                              // selects (1); 0: match.any
#endif
#ifndef K3_BLOCK_CFG
#define K3_BLOCK_CFG 256
#endif
#ifndef K3_WINDOW_CFG
#define K3_WINDOW_CFG 8
#endif
#ifndef K3_CLAIM_CFG
#define K3_CLAIM_CFG 1        // when a block claims its next tile: 0 while starting the current one,
                              // 1 when it starts the next one, 2 after the current look-back
#endif
constexpr int K3_BLOCK = K3_BLOCK_CFG;
constexpr int K3_WARPS = K3_BLOCK / 32;
constexpr int K3_ITEMS = K3_ITEMS_CFG;
constexpr int K3_TILE = K3_BLOCK * K3_ITEMS;
constexpr int K3_WARP_ITEMS = 32 * K3_ITEMS;
constexpr int K3_WINDOW = K3_WINDOW_CFG;          // status words in flight per look-back step
static_assert(K3_BLOCK == kRadix || K3_BLOCK == 2 * kRadix, "the first kRadix threads own a digit each");
static_assert(K3_WARP_ITEMS <= 65535, "16-bit warp counters");

__device__ __forceinline__ u32 digit_of(u64 k, u32 shift) { return (u32)(k >> shift) & (kRadix - 1); }

// Digit of pass P: a bit-field extract from one 32-bit half of the key.
template <int P>
__device__ __forceinline__ u32 digit_p(u64 k) {
  if (P >= kMaxPasses) return 0u;
  const u32 half = P < 4 ? (u32)k : (u32)(k >> 32);
  return (half >> ((P & 3) * kRadixBits)) & (kRadix - 1);
}

// Lanes holding the same 8-bit digit (all 32 lanes take part).
__device__ __forceinline__ u32 same_digit_lanes(u32 dg) {
#if K3_RANK_BALLOT == 3
  return warp_digit_peers(dg);
#elif K3_RANK_BALLOT == 2
  // A lane differs from this one where some ballot differs from this
  // lane's own bit (replicated to a full mask).
  u32 differ = 0u;
  #pragma unroll
  for (int b = 0; b < kRadixBits; ++b) {
    const u32 mine = 0u - ((dg >> b) & 1u);
    differ |= __ballot_sync(0xFFFFFFFFu, mine != 0u) ^ mine;
  }
  return ~differ;
#elif K3_RANK_BALLOT
  u32 peers = 0xFFFFFFFFu;
  #pragma unroll
  for (int b = 0; b < kRadixBits; ++b) {
    const bool bit = (dg >> b) & 1u;
    const u32 bal = __ballot_sync(0xFFFFFFFFu, bit);
    peers &= bit ? bal : ~bal;
  }
  return peers;
#else
  return __match_any_sync(0xFFFFFFFFu, dg);
#endif
}

template <int PASS>
__global__ void __launch_bounds__(K3_BLOCK, K3_MINBLOCKS_CFG)
k3_onesweep(const u64* __restrict__ keys_in, const u32* __restrict__ idx_in,
            u64* __restrict__ keys_out, u32* __restrict__ idx_out, Plan* plan,
            u64* __restrict__ status) {
  constexpr u32 pass = PASS;
  extern __shared__ __align__(16) unsigned char k3_smem[];
  u64* s_keys = reinterpret_cast<u64*>(k3_smem);
  u32* s_idx = reinterpret_cast<u32*>(k3_smem + K3_TILE * sizeof(u64));
  // Per-warp digit counts, then each warp's next free tile position per digit.
  __shared__ u32 s_wpos[K3_WARPS][kRadix];
  __shared__ u32 s_next[kRadix];      // next pass's digit histogram (block lifetime)
  __shared__ u32 s_gstart[kRadix];
  __shared__ u32 s_gbase[kRadix];
  __shared__ u32 s_warp_tot[kRadix / 32];
  __shared__ u32 s_tile[2];
  __shared__ int s_fail;

  const u32 npasses = plan->npasses;
  if (pass >= npasses || (plan->error & ERR_RANGE)) return;
  const u32 s = plan->s;
  const bool count_next = pass + 1 < npasses;
  const u32 epoch = plan->epoch + EP_SORT0 + pass;
  const u32 spin = plan->spin_limit;
  const u32 ntiles = (s + K3_TILE - 1) / K3_TILE;
  const int d = threadIdx.x & (kRadix - 1);      // digit owned in the per-digit phases
  const bool owner = threadIdx.x < kRadix;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const u32 lt_mask = (1u << lane) - 1u;
  u32* ctr = &plan->ctr[CTR_SORT0 + pass];

  // Global exclusive start of every digit (scan of the histogram by the
  // digit owners).
  u32 hv = 0, hinc = 0;
  if (owner) {
    hv = plan->hist[pass][d];
    hinc = hv;
    #pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const u32 t = __shfl_up_sync(0xFFFFFFFFu, hinc, o);
      if (lane >= o) hinc += t;
    }
    if (lane == 31) s_warp_tot[wid] = hinc;
    s_next[d] = 0;
  }
  if (K3_CLAIM_CFG != 1 && threadIdx.x == 0) s_tile[0] = atomicAdd(ctr, 1u);
  __syncthreads();
  if (owner) {
    u32 off = 0;
    for (int w = 0; w < wid; ++w) off += s_warp_tot[w];
    s_gstart[d] = off + hinc - hv;
  }

  for (int buf = 0;; buf ^= 1) {
    if (K3_CLAIM_CFG == 1 && threadIdx.x == 0) s_tile[buf] = atomicAdd(ctr, 1u);
    for (int q = threadIdx.x; q < K3_WARPS * kRadix; q += K3_BLOCK) (&s_wpos[0][0])[q] = 0u;
    __syncthreads();
    const u32 tile = s_tile[buf];
    if (tile >= ntiles) break;
    if (K3_CLAIM_CFG == 0 && threadIdx.x == 0) s_tile[buf ^ 1] = atomicAdd(ctr, 1u);
    const u32 base = tile * (u32)K3_TILE;
    const u32 tile_n = min((u32)K3_TILE, s - base);
    const bool full = tile_n == (u32)K3_TILE;

    u64 key[K3_ITEMS];
    u32 idv[K3_ITEMS];
    const u32 wbase = base + wid * K3_WARP_ITEMS;
    #pragma unroll
    for (int it = 0; it < K3_ITEMS; ++it) {
      const u32 p = wbase + it * 32 + lane;
      const bool v = full || p < s;
      key[it] = v ? keys_in[p] : 0ull;
      idv[it] = v ? idx_in[p] : 0u;
    }
    // Per-warp digit counts (and the next pass's histogram).
    u32* wp = &s_wpos[wid][0];
    #pragma unroll
    for (int it = 0; it < K3_ITEMS; ++it) {
      if (full || wbase + it * 32 + lane < s) {
        atomicAdd(&wp[digit_p<PASS>(key[it])], 1u);
        if (count_next) atomicAdd(&s_next[digit_p<PASS + 1>(key[it])], 1u);
      }
    }
    __syncthreads();
    // Per digit: tile count (published at once), tile-local start, and each
    // warp's first position.
    u32 cnt = 0, tinc = 0;
    u64* st = status + (size_t)tile * kRadix + d;
    if (owner) {
      #pragma unroll
      for (int w = 0; w < K3_WARPS; ++w) cnt += s_wpos[w][d];
      st_relaxed_u64(st, make_status(epoch, tile == 0 ? ST_INCL : ST_AGG, cnt));
      tinc = cnt;
      #pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const u32 t = __shfl_up_sync(0xFFFFFFFFu, tinc, o);
        if (lane >= o) tinc += t;
      }
      if (lane == 31) s_warp_tot[wid] = tinc;
    }
    __syncthreads();
    u32 tstart = 0;
    if (owner) {
      u32 off = 0;
      for (int w = 0; w < wid; ++w) off += s_warp_tot[w];
      tstart = off + tinc - cnt;
      u32 run = tstart;
      #pragma unroll
      for (int w = 0; w < K3_WARPS; ++w) {
        const u32 c = s_wpos[w][d];
        s_wpos[w][d] = run;
        run += c;
      }
    }
    __syncthreads();

    // Stable ranking, item by item in input order, straight into the tile's
    // digit-ordered staging area: the highest lane of each group of equal
    // digits reserves the group's positions with one shared atomic.
    #pragma unroll
    for (int it = 0; it < K3_ITEMS; ++it) {
      const u32 dg = digit_p<PASS>(key[it]);
      const bool valid = full || (wbase + it * 32 + lane) < s;
      u32 peers = same_digit_lanes(dg);
      if (!full) peers &= __ballot_sync(0xFFFFFFFFu, valid);
      const int leader = 31 - __clz(peers);
      u32 pos = 0;
      if (valid && lane == leader) pos = atomicAdd(&wp[dg], (u32)__popc(peers));
      pos = __shfl_sync(0xFFFFFFFFu, pos, valid ? leader : lane) + __popc(peers & lt_mask);
      if (valid) {
        s_keys[pos] = key[it];
        s_idx[pos] = idv[it];
      }
    }

    // Decoupled look-back for this digit, K3_WINDOW predecessors per step.
    u32 excl = 0;
    bool fail = false;
    if (owner) {
      if (tile > 0) {
        long long t = (long long)tile - 1;
        bool done = false;
        while (!done && !fail) {
          u64 w[K3_WINDOW];
          #pragma unroll
          for (int k = 0; k < K3_WINDOW; ++k)
            w[k] = (t - k >= 0) ? ld_relaxed_u64(status + (size_t)(t - k) * kRadix + d)
                                : make_status(epoch, ST_INCL, 0);
          #pragma unroll
          for (int k = 0; k < K3_WINDOW; ++k) {
            if (done || fail) break;
            u32 f = status_flag(w[k], epoch);
            u32 it = 0;
            while (f == 0) {
              if (++it > spin || aborted(plan)) { fail = true; break; }
              spin_pause(it);
              w[k] = ld_relaxed_u64(status + (size_t)(t - k) * kRadix + d);
              f = status_flag(w[k], epoch);
            }
            if (fail) break;
            excl += status_count(w[k]);
            if (f == ST_INCL) done = true;
          }
          t -= K3_WINDOW;
        }
        if (!fail) st_relaxed_u64(st, make_status(epoch, ST_INCL, excl + cnt));
      }
      if (fail) flag_error(plan, ERR_TIMEOUT);
      s_gbase[d] = s_gstart[d] + excl - tstart;
    }
    // A tile claimed before its block can start it holds up its successors'
    // look-backs until it starts (mode 0 claims a whole tile ahead).
    if (K3_CLAIM_CFG == 2 && threadIdx.x == 0) s_tile[buf ^ 1] = atomicAdd(ctr, 1u);
    if (threadIdx.x == 0) s_fail = 0;
    __syncthreads();
    if (fail) s_fail = 1;
    __syncthreads();
    if (s_fail) break;

    // Write the digit-ordered tile out: consecutive threads, consecutive
    // addresses within each digit.
    if (full) {
      #pragma unroll
      for (int it = 0; it < K3_ITEMS; ++it) {
        const u32 j = it * K3_BLOCK + threadIdx.x;
        const u64 k = s_keys[j];
        const u32 gp = s_gbase[digit_p<PASS>(k)] + j;
        if (gp < s) {
          keys_out[gp] = k;
          idx_out[gp] = s_idx[j];
        } else {
          flag_error(plan, ERR_INTERNAL);
        }
      }
    } else {
      for (u32 j = threadIdx.x; j < tile_n; j += K3_BLOCK) {
        const u64 k = s_keys[j];
        const u32 gp = s_gbase[digit_p<PASS>(k)] + j;
        if (gp < s) {
          keys_out[gp] = k;
          idx_out[gp] = s_idx[j];
        } else {
          flag_error(plan, ERR_INTERNAL);
        }
      }
    }
  }
  if (count_next && owner) {
    const u32 c = s_next[d];
    if (c) atomicAdd(&plan->hist[pass + 1][d], c);
  }
}

}  // namespace

int k3_tile() { return K3_TILE; }
size_t k3_dyn_smem() { return (size_t)K3_TILE * (sizeof(u64) + sizeof(u32)); }

template <int P>
static cudaError_t configure_pass() {
  return cudaFuncSetAttribute(k3_onesweep<P>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)k3_dyn_smem());
}

cudaError_t k3_configure() {
  cudaError_t e = configure_pass<0>();
  if (e == cudaSuccess) e = configure_pass<1>();
  if (e == cudaSuccess) e = configure_pass<2>();
  if (e == cudaSuccess) e = configure_pass<3>();
  if (e == cudaSuccess) e = configure_pass<4>();
  if (e == cudaSuccess) e = configure_pass<5>();
  if (e == cudaSuccess) e = configure_pass<6>();
  if (e == cudaSuccess) e = configure_pass<7>();
  return e;
}

cudaError_t k3_occupancy(int* blocks) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, k3_onesweep<0>, K3_BLOCK, k3_dyn_smem());
}

cudaError_t launch_k3(const u64* kin, const u32* iin, u64* kout, u32* iout, Plan* plan,
                      u64* status, u32 pass, int grid, cudaStream_t st) {
  const size_t sm = k3_dyn_smem();
  switch (pass) {
    case 0: k3_onesweep<0><<<grid, K3_BLOCK, sm, st>>>(kin, iin, kout, iout, plan, status); break;
    case 1: k3_onesweep<1><<<grid, K3_BLOCK, sm, st>>>(kin, iin, kout, iout, plan, status); break;
    case 2: k3_onesweep<2><<<grid, K3_BLOCK, sm, st>>>(kin, iin, kout, iout, plan, status); break;
    case 3: k3_onesweep<3><<<grid, K3_BLOCK, sm, st>>>(kin, iin, kout, iout, plan, status); break;
    case 4: k3_onesweep<4><<<grid, K3_BLOCK, sm, st>>>(kin, iin, kout, iout, plan, status); break;
    case 5: k3_onesweep<5><<<grid, K3_BLOCK, sm, st>>>(kin, iin, kout, iout, plan, status); break;
    case 6: k3_onesweep<6><<<grid, K3_BLOCK, sm, st>>>(kin, iin, kout, iout, plan, status); break;
    case 7: k3_onesweep<7><<<grid, K3_BLOCK, sm, st>>>(kin, iin, kout, iout, plan, status); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace gbh
