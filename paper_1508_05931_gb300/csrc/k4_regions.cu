// K4: region split and the second-round filter (Section 2.1 steps 5-7,
// Section 2.2 / Figure 2, Section 3.4), fused with the stable compaction
// that Section 3.4 performs with a stable partition.
//
// Over the sorted survivors: P_0 = P_minx (first in the lexicographic
// order) and P_l = P_maxx (the last distinct point, its smallest index).
// A point strictly right of the directed line P_0 -> P_l belongs to the
// lower region, strictly left to the upper region; points on the line are
// dropped.  Figure 2 walks a region with a running P_temp and discards P_i
// when it lies left of (right of, for the upper region) or on the line
// P_temp -> P_l.  With d(p) = p - P_l, that rule keeps P_i exactly when
// d(P_i) is strictly counter-clockwise (clockwise) of d(P_temp), and P_temp
// is always the point with the extreme direction seen so far, starting from
// d(P_0).  All directions of a region lie in one half-plane, where the
// cross product orders them totally, so "extreme so far" is an exclusive
// prefix max (min) -- an associative scan.  It is computed here with one
// decoupled look-back and gives exactly the survivors of the sequential
// loop, for any tile size; duplicates of a kept point fall out as equal
// directions.  Kept points are compacted stably per region with a second
// look-back chained behind the first; the last tile adds P_0 and P_l.
#include "hull_internal.cuh"
#include "kernels.h"

namespace gbh {

namespace {

constexpr int K4_BLOCK = 256;
constexpr int K4_ITEMS = 16;
constexpr int K4_TILE = K4_BLOCK * K4_ITEMS;
constexpr int K4_WARPS = K4_BLOCK / 32;

constexpr u32 K4_AGG = 1, K4_DIRP = 2, K4_FULL = 3;

struct __align__(64) K4Status {
  u64 flag;                 // [epoch:32 | state:32]
  int agg[4];               // tile aggregate: lower max dir (x,y), upper min dir (x,y)
  int inc[4];               // inclusive prefix of the same
  u32 cnt[2];               // kept counts of this tile (lower, upper)
  u32 inc_cnt[2];           // inclusive kept counts
};
static_assert(sizeof(K4Status) == 64, "status record size");

// Direction pairs; (0, 0) marks "no element".
struct Dir2 {
  int lx, ly, ux, uy;
};

__device__ __forceinline__ bool is_empty(int x, int y) { return (x | y) == 0; }

// Lower region: keep the counter-clockwise-most direction (ties keep a).
__device__ __forceinline__ void cmax(int& ax, int& ay, int bx, int by) {
  if (is_empty(bx, by)) return;
  if (is_empty(ax, ay) || cross2(ax, ay, bx, by) > 0) { ax = bx; ay = by; }
}
// Upper region: keep the clockwise-most direction (ties keep a).
__device__ __forceinline__ void cmin(int& ax, int& ay, int bx, int by) {
  if (is_empty(bx, by)) return;
  if (is_empty(ax, ay) || cross2(ax, ay, bx, by) < 0) { ax = bx; ay = by; }
}
__device__ __forceinline__ void combine(Dir2& a, const Dir2& b) {
  cmax(a.lx, a.ly, b.lx, b.ly);
  cmin(a.ux, a.uy, b.ux, b.uy);
}
__device__ __forceinline__ Dir2 shfl_up_dir(const Dir2& v, int o) {
  Dir2 r;
  r.lx = __shfl_up_sync(0xFFFFFFFFu, v.lx, o);
  r.ly = __shfl_up_sync(0xFFFFFFFFu, v.ly, o);
  r.ux = __shfl_up_sync(0xFFFFFFFFu, v.ux, o);
  r.uy = __shfl_up_sync(0xFFFFFFFFu, v.uy, o);
  return r;
}

__device__ __forceinline__ u32 wait_state(const K4Status* st, u32 epoch, u32 need, u32 spin,
                                          Plan* plan, bool* fail) {
  u32 it = 0;
  for (;;) {
    u64 w = ld_acquire_u64(&st->flag);
    u32 state = ((u32)(w >> 32) == epoch) ? (u32)w : 0u;
    if (state >= need) return state;
    if (++it > spin || aborted(plan)) { *fail = true; return 0; }
    spin_pause(it);
  }
}

__global__ void __launch_bounds__(K4_BLOCK)
k4_regions(const u64* __restrict__ keys_a, const u32* __restrict__ idx_a,
           const u64* __restrict__ keys_b, const u32* __restrict__ idx_b, Plan* plan,
           K4Status* __restrict__ status, int2* __restrict__ lo_xy, int* __restrict__ lo_idx,
           int2* __restrict__ up_xy, int* __restrict__ up_idx) {
  __shared__ Dir2 s_wdir[K4_WARPS];
  __shared__ u32 s_wcnt[K4_WARPS][2];
  __shared__ Dir2 s_tile_excl;
  __shared__ u32 s_cnt_excl[2];
  __shared__ u32 s_tile;
  __shared__ int s_fail;

  if (plan->error & ERR_RANGE) return;
  // The sort leaves its result in buffer a after an even number of passes.
  const bool in_b = (plan->npasses & 1u) != 0;
  const u64* __restrict__ keys = in_b ? keys_b : keys_a;
  const u32* __restrict__ idxs = in_b ? idx_b : idx_a;
  const u32 s = plan->s;
  const u32 epoch = plan->epoch + EP_REGION;
  const u32 spin = plan->spin_limit;
  const u32 ybits = plan->ybits;
  const u64 ymask = ybits ? ((~0ull) >> (64 - ybits)) : 0ull;
  const int x0 = plan->key_x0, y0 = plan->key_y0;
  const int ax = plan->ext_x[0], ay = plan->ext_y[0];     // P_0 = P_minx
  const int bx = plan->ext_x[1], by = plan->ext_y[1];     // P_l = P_maxx
  const int ux = bx - ax, uy = by - ay;
  const int d0x = ax - bx, d0y = ay - by;                 // d(P_0)
  const u32 ntiles = (s + K4_TILE - 1) / K4_TILE;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;

  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) s_tile = atomicAdd(&plan->ctr[CTR_REGION], 1u);
    __syncthreads();
    const u32 tile = s_tile;
    if (tile >= ntiles) break;
    const u32 first = tile * (u32)K4_TILE + threadIdx.x * K4_ITEMS;

    // Blocked arrangement: this thread owns K4_ITEMS consecutive items.
    int px[K4_ITEMS], py[K4_ITEMS], pi[K4_ITEMS];
    signed char side[K4_ITEMS];
    #pragma unroll
    for (int i = 0; i < K4_ITEMS; ++i) {
      const u32 p = first + i;
      side[i] = 0;
      px[i] = 0; py[i] = 0; pi[i] = 0;
      if (p < s) {
        const u64 k = keys[p];
        px[i] = x0 + (int)(u32)(k >> ybits);
        py[i] = y0 + (int)(u32)(k & ymask);
        pi[i] = (int)idxs[p];
        const long long o = cross2(ux, uy, px[i] - ax, py[i] - ay);
        side[i] = (o < 0) ? -1 : (o > 0 ? 1 : 0);
      }
    }
    Dir2 agg = {0, 0, 0, 0};
    #pragma unroll
    for (int i = 0; i < K4_ITEMS; ++i) {
      if (side[i] < 0) cmax(agg.lx, agg.ly, px[i] - bx, py[i] - by);
      else if (side[i] > 0) cmin(agg.ux, agg.uy, px[i] - bx, py[i] - by);
    }
    // Warp inclusive scan of the thread aggregates.
    Dir2 inc = agg;
    #pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      Dir2 t = shfl_up_dir(inc, o);
      if (lane >= o) {
        Dir2 r = t;
        combine(r, inc);
        inc = r;
      }
    }
    Dir2 lane_excl = shfl_up_dir(inc, 1);
    if (lane == 0) lane_excl = Dir2{0, 0, 0, 0};
    if (lane == 31) s_wdir[wid] = inc;
    __syncthreads();

    // Tile aggregate, publish, look-back over directions.
    if (threadIdx.x == 0) {
      Dir2 tagg = {0, 0, 0, 0};
      for (int w = 0; w < K4_WARPS; ++w) combine(tagg, s_wdir[w]);
      K4Status* me = &status[tile];
      bool fail = false;
      Dir2 excl = {d0x, d0y, d0x, d0y};
      if (tile > 0) {
        me->agg[0] = tagg.lx; me->agg[1] = tagg.ly; me->agg[2] = tagg.ux; me->agg[3] = tagg.uy;
        st_release_u64(&me->flag, ((u64)epoch << 32) | K4_AGG);
        Dir2 acc = {0, 0, 0, 0};
        for (long long t = (long long)tile - 1; t >= 0; --t) {
          const volatile K4Status* o = &status[t];
          u32 stt = wait_state(&status[t], epoch, K4_AGG, spin, plan, &fail);
          if (fail) break;
          if (stt >= K4_DIRP) {
            Dir2 v = {o->inc[0], o->inc[1], o->inc[2], o->inc[3]};
            combine(acc, v);
            break;
          }
          Dir2 v = {o->agg[0], o->agg[1], o->agg[2], o->agg[3]};
          combine(acc, v);
        }
        excl = acc;
      }
      if (fail) flag_error(plan, ERR_TIMEOUT);
      s_tile_excl = excl;
      s_fail = fail ? 1 : 0;
    }
    __syncthreads();
    if (s_fail) break;

    // This thread's exclusive prefix and the keep decisions.
    Dir2 run = s_tile_excl;
    for (int w = 0; w < wid; ++w) combine(run, s_wdir[w]);
    combine(run, lane_excl);
    unsigned keep_lo = 0, keep_up = 0;
    #pragma unroll
    for (int i = 0; i < K4_ITEMS; ++i) {
      const int vx = px[i] - bx, vy = py[i] - by;
      if (side[i] < 0) {
        if (cross2(run.lx, run.ly, vx, vy) > 0) { keep_lo |= 1u << i; run.lx = vx; run.ly = vy; }
      } else if (side[i] > 0) {
        if (cross2(run.ux, run.uy, vx, vy) < 0) { keep_up |= 1u << i; run.ux = vx; run.uy = vy; }
      }
    }
    // Stable ranks of the kept points (block scan of two counts).
    u32 c_lo = __popc(keep_lo), c_up = __popc(keep_up);
    u32 i_lo = c_lo, i_up = c_up;
    #pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      u32 t0 = __shfl_up_sync(0xFFFFFFFFu, i_lo, o);
      u32 t1 = __shfl_up_sync(0xFFFFFFFFu, i_up, o);
      if (lane >= o) { i_lo += t0; i_up += t1; }
    }
    if (lane == 31) { s_wcnt[wid][0] = i_lo; s_wcnt[wid][1] = i_up; }
    __syncthreads();
    if (threadIdx.x == 0) {
      u32 tl = 0, tu = 0;
      for (int w = 0; w < K4_WARPS; ++w) {
        u32 a0 = s_wcnt[w][0], a1 = s_wcnt[w][1];
        s_wcnt[w][0] = tl; s_wcnt[w][1] = tu;
        tl += a0; tu += a1;
      }
      K4Status* me = &status[tile];
      Dir2 tinc = s_tile_excl;
      Dir2 tagg = {0, 0, 0, 0};
      for (int w = 0; w < K4_WARPS; ++w) combine(tagg, s_wdir[w]);
      combine(tinc, tagg);
      me->inc[0] = tinc.lx; me->inc[1] = tinc.ly; me->inc[2] = tinc.ux; me->inc[3] = tinc.uy;
      me->cnt[0] = tl; me->cnt[1] = tu;
      bool fail = false;
      u32 e_lo = 0, e_up = 0;
      if (tile == 0) {
        me->inc_cnt[0] = tl; me->inc_cnt[1] = tu;
        st_release_u64(&me->flag, ((u64)epoch << 32) | K4_FULL);
      } else {
        st_release_u64(&me->flag, ((u64)epoch << 32) | K4_DIRP);
        for (long long t = (long long)tile - 1; t >= 0; --t) {
          const volatile K4Status* o = &status[t];
          u32 stt = wait_state(&status[t], epoch, K4_DIRP, spin, plan, &fail);
          if (fail) break;
          if (stt == K4_FULL) { e_lo += o->inc_cnt[0]; e_up += o->inc_cnt[1]; break; }
          e_lo += o->cnt[0]; e_up += o->cnt[1];
        }
        if (!fail) {
          me->inc_cnt[0] = e_lo + tl; me->inc_cnt[1] = e_up + tu;
          st_release_u64(&me->flag, ((u64)epoch << 32) | K4_FULL);
        }
      }
      if (fail) flag_error(plan, ERR_TIMEOUT);
      s_fail = fail ? 1 : 0;
      s_cnt_excl[0] = e_lo;
      s_cnt_excl[1] = e_up;
      if (tile == ntiles - 1 && !fail) {
        const u32 r_lo = e_lo + tl, r_up = e_up + tu;
        plan->r_lo = r_lo;
        plan->r_up = r_up;
        const int ia = plan->ext_idx[0], ib = plan->ext_idx[1];
        lo_xy[0] = make_int2(ax, ay); lo_idx[0] = ia;
        up_xy[0] = make_int2(ax, ay); up_idx[0] = ia;
        if (r_lo + 1 < s + 2) { lo_xy[r_lo + 1] = make_int2(bx, by); lo_idx[r_lo + 1] = ib; }
        if (r_up + 1 < s + 2) { up_xy[r_up + 1] = make_int2(bx, by); up_idx[r_up + 1] = ib; }
      }
    }
    __syncthreads();
    if (s_fail) break;
    u32 pos_lo = 1 + s_cnt_excl[0] + s_wcnt[wid][0] + (i_lo - c_lo);
    u32 pos_up = 1 + s_cnt_excl[1] + s_wcnt[wid][1] + (i_up - c_up);
    #pragma unroll
    for (int i = 0; i < K4_ITEMS; ++i) {
      if (keep_lo & (1u << i)) {
        if (pos_lo < s + 1) { lo_xy[pos_lo] = make_int2(px[i], py[i]); lo_idx[pos_lo] = pi[i]; }
        else flag_error(plan, ERR_INTERNAL);
        ++pos_lo;
      } else if (keep_up & (1u << i)) {
        if (pos_up < s + 1) { up_xy[pos_up] = make_int2(px[i], py[i]); up_idx[pos_up] = pi[i]; }
        else flag_error(plan, ERR_INTERNAL);
        ++pos_up;
      }
    }
  }
}

}  // namespace

int k4_tile() { return K4_TILE; }

cudaError_t k4_occupancy(int* blocks) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, k4_regions, K4_BLOCK, 0);
}
size_t k4_status_bytes() { return sizeof(K4Status); }

cudaError_t launch_k4(const u64* ka, const u32* ia, const u64* kb, const u32* ib, Plan* plan,
                      void* status, int2* lo_xy, int* lo_idx, int2* up_xy, int* up_idx, int grid,
                      cudaStream_t st) {
  k4_regions<<<grid, K4_BLOCK, 0, st>>>(ka, ia, kb, ib, plan, reinterpret_cast<K4Status*>(status),
                                        lo_xy, lo_idx, up_xy, up_idx);
  return cudaGetLastError();
}

}  // namespace gbh
