// K5: the finalisation (Section 2.1 step 8; Sections 3 and 5.2 run it on
// the CPU as a stack-based scan of the pre-sorted survivors).  Here it runs
// on the device as a parallel monotone chain:
//
//   phase A  each block takes chunks of C consecutive points of a chain
//            (C the smallest power of two from K5_MIN_CHUNK to K5_CHUNK that
//            gives every block at most one chunk: short lists are spread
//            over many SMs and every chunk's merge tree stays shallow);
//            every thread builds the chain of its K5_LEAF points with
//            the stack rule (pop while the turn is not strict), and adjacent
//            sub-chains are merged level by level in shared memory (one
//            thread per pair while they are short, then one warp per pair);
//   phase B  when all chunk chains together fit in one block's shared
//            memory (the usual case: a chunk's chain holds few of its
//            points), block 0 gathers them after one grid barrier and merges
//            them there level by level; otherwise adjacent chunk chains are
//            merged level by level across the grid (ping-pong buffers,
//            bounded grid barriers);
//   output   lower chain, then the upper chain reversed without its two
//            endpoints: counter-clockwise from the lexicographic minimum.
//
// The merge of two adjacent chains at their common tangent is described in
// chain.cuh.
#include <cooperative_groups.h>

#include "chain.cuh"
#include "hull_internal.cuh"
#include "kernels.h"

namespace gbh {

using namespace chain;

namespace {

#ifndef K5_BLOCK_CFG
#define K5_BLOCK_CFG 1024
#endif
constexpr int K5_BLOCK = K5_BLOCK_CFG;
constexpr int K5_WARPS = K5_BLOCK / 32;
#ifndef K5_LEAF_CFG
#define K5_LEAF_CFG 2
#endif
constexpr int K5_LEAF = K5_LEAF_CFG;
constexpr int K5_CHUNK = K5_BLOCK * K5_LEAF;   // points per chunk, at most
#ifndef K5_MIN_CHUNK_CFG
#define K5_MIN_CHUNK_CFG 256
#endif
constexpr int K5_MIN_CHUNK = K5_MIN_CHUNK_CFG;   // points per chunk, at least
// Points block 0 can hold for the shared-memory phase B (and the size of
// every block's chunk buffer).
constexpr int K5_SMEM_PTS = K5_CHUNK > 16384 ? K5_CHUNK : 16384;

// Barrier over the first `nblocks` blocks of the (co-resident) grid.
__device__ bool grid_barrier(Plan* plan, u32 spin, u32 nblocks) {
  __syncthreads();
  __shared__ int s_bar_fail;
  if (threadIdx.x == 0) {
    s_bar_fail = 0;
    __threadfence();
    volatile u32* genp = &plan->ctr[CTR_FINAL_BAR_GEN];
    const u32 gen = *genp;
    const u32 arrived = atomicAdd(&plan->ctr[CTR_FINAL_BAR], 1u) + 1u;
    if (arrived == nblocks) {
      plan->ctr[CTR_FINAL_BAR] = 0u;
      __threadfence();
      atomicAdd(&plan->ctr[CTR_FINAL_BAR_GEN], 1u);
    } else {
      u32 it = 0;
      while (*genp == gen) {
        if (++it > spin || aborted(plan)) {
          flag_error(plan, ERR_TIMEOUT);
          s_bar_fail = 1;
          break;
        }
        spin_pause(it);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return s_bar_fail == 0;
}

struct ChainSet {
  const int2* in_xy[2];
  const int* in_idx[2];
  u32 m[2];          // points per chain
  u32 nchunk[2];
  u32 slot0[2];      // first slot of each chain in the ping-pong buffers
};

__global__ void __launch_bounds__(K5_BLOCK)
k5_final(const int2* __restrict__ lo_xy, const int* __restrict__ lo_idx,
         const int2* __restrict__ up_xy, const int* __restrict__ up_idx, Plan* plan,
         int2* __restrict__ h0_xy, int* __restrict__ h0_idx, int2* __restrict__ h1_xy,
         int* __restrict__ h1_idx, u32* __restrict__ cnt0, u32* __restrict__ cnt1,
         int4* __restrict__ jobs, int* __restrict__ out, long long cap) {
  extern __shared__ __align__(16) unsigned char k5_smem[];
  int* sx = reinterpret_cast<int*>(k5_smem);
  int* sy = sx + K5_SMEM_PTS;
  int* si = sy + K5_SMEM_PTS;
  __shared__ int s_cnt[K5_BLOCK];
  __shared__ int s_start[K5_BLOCK];
  __shared__ int s_wsum[K5_WARPS];
  __shared__ int4 s_pair[K5_BLOCK / 2 + 1];

  if (plan->error & (ERR_RANGE | ERR_TIMEOUT | ERR_INTERNAL | ERR_FALLBACK)) return;
  const u32 spin = plan->spin_limit;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;

  ChainSet cs;
  cs.in_xy[0] = lo_xy; cs.in_idx[0] = lo_idx;
  cs.in_xy[1] = up_xy; cs.in_idx[1] = up_idx;
  cs.m[0] = plan->r_lo + 2;
  cs.m[1] = plan->r_up + 2;
  u32 C = K5_MIN_CHUNK;
  while (C < (u32)K5_CHUNK && (cs.m[0] + C - 1) / C + (cs.m[1] + C - 1) / C > gridDim.x) C <<= 1;
  for (int c = 0; c < 2; ++c) cs.nchunk[c] = (cs.m[c] + C - 1) / C;
  cs.slot0[0] = 0;
  cs.slot0[1] = cs.nchunk[0] * C;

  // Every point equal: the hull is the single point P_0.
  {
    const int2 a = lo_xy[0], b = lo_xy[cs.m[0] - 1];
    if (cs.m[0] == 2 && cs.m[1] == 2 && a.x == b.x && a.y == b.y) {
      if (blockIdx.x == 0 && threadIdx.x == 0) {
        plan->h = 1; plan->h_lo = 1; plan->h_up = 1;
        if (cap >= 1) out[0] = lo_idx[0];
        else flag_error(plan, ERR_CAPACITY);
      }
      return;
    }
  }

  // Only as many blocks as the work needs take part (the same count on
  // every block: it depends only on the Plan); the others leave now.
  const u32 total_chunks = cs.nchunk[0] + cs.nchunk[1];
  const u32 nblk = min(gridDim.x, max(16u, total_chunks));
  if (blockIdx.x >= nblk) return;

  // ---------------- phase A: chunk chains in shared memory
  for (u32 ch = blockIdx.x; ch < total_chunks; ch += nblk) {
    const int c = ch < cs.nchunk[0] ? 0 : 1;
    const u32 local = c == 0 ? ch : ch - cs.nchunk[0];
    const int sgn = c == 0 ? 1 : -1;
    const u32 first = local * C;
    const int len = (int)min(C, cs.m[c] - first);
    for (int i = threadIdx.x; i < len; i += K5_BLOCK) {
      const int2 p = cs.in_xy[c][first + i];
      sx[i] = p.x; sy[i] = p.y; si[i] = cs.in_idx[c][first + i];
    }
    __syncthreads();
    {
      const int b = threadIdx.x * K5_LEAF;
      s_cnt[threadIdx.x] = leaf_chain(sx, sy, si, b, max(0, min(K5_LEAF, len - b)), sgn);
    }
    __syncthreads();
    const int nleaf = (len + K5_LEAF - 1) / K5_LEAF;
    merge_tree<K5_LEAF>(sx, sy, si, s_cnt, s_pair, nleaf, sgn);
    const int hc = s_cnt[0];
    const u32 out0 = cs.slot0[c] + first;
    for (int i = threadIdx.x; i < hc; i += K5_BLOCK) {
      h0_xy[out0 + i] = make_int2(sx[i], sy[i]);
      h0_idx[out0 + i] = si[i];
    }
    if (threadIdx.x == 0) cnt0[cs.slot0[c] / C + local] = (u32)hc;
    __syncthreads();
  }

  // ---------------- phase B, small case: one block, shared memory
  if (!grid_barrier(plan, spin, nblk)) return;
  if (total_chunks <= (u32)K5_BLOCK) {
    // Chunk chain lengths and their exclusive prefix (same on every block).
    const int len_c = threadIdx.x < total_chunks ? (int)__ldcg(&cnt0[threadIdx.x]) : 0;
    int inc = len_c;
    #pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xFFFFFFFFu, inc, o);
      if (lane >= o) inc += t;
    }
    if (lane == 31) s_wsum[wid] = inc;
    __syncthreads();
    int off = 0, tot = 0;
    for (int w = 0; w < K5_WARPS; ++w) {
      if (w < wid) off += s_wsum[w];
      tot += s_wsum[w];
    }
    if (tot <= K5_SMEM_PTS) {
      if (blockIdx.x != 0) return;
      s_cnt[threadIdx.x] = len_c;
      s_start[threadIdx.x] = off + inc - len_c;
      __syncthreads();
      // Gather: warp w copies chunk chains w, w + K5_WARPS, ...
      for (u32 ch = wid; ch < total_chunks; ch += K5_WARPS) {
        const u32 src = ch < cs.nchunk[0] ? ch * C : cs.slot0[1] + (ch - cs.nchunk[0]) * C;
        const int dst = s_start[ch];
        for (int q = lane; q < s_cnt[ch]; q += 32) {
          const int2 p = __ldcg(&h0_xy[src + q]);
          sx[dst + q] = p.x; sy[dst + q] = p.y; si[dst + q] = __ldcg(&h0_idx[src + q]);
        }
      }
      __syncthreads();
      // Merge both regions' chains level by level (one warp per pair).
      const int n0 = (int)cs.nchunk[0], n1 = (int)cs.nchunk[1];
      for (int step = 1; step < max(n0, n1); step <<= 1) {
        const int np0 = (n0 + 2 * step - 1) / (2 * step), np1 = (n1 + 2 * step - 1) / (2 * step);
        for (int job = wid; job < np0 + np1; job += K5_WARPS) {
          const int c = job < np0 ? 0 : 1;
          const int p = c == 0 ? job : job - np0;
          const int k0 = c == 0 ? 0 : n0, kn = c == 0 ? n0 : n1;
          const int a = 2 * p * step, b = a + step;
          if (b >= kn) continue;
          const int ka = k0 + a, kb = k0 + b;
          const int alpha = s_cnt[ka], beta = s_cnt[kb];
          SmemChain A{sx + s_start[ka], sy + s_start[ka]}, B{sx + s_start[kb], sy + s_start[kb]};
          int is, js;
          bridge(A, alpha, B, beta, c == 0 ? 1 : -1, is, js);
          const int dst = s_start[ka] + is + 1, src = s_start[kb] + js, n2 = beta - js;
          for (int o = 0; o < n2; o += 32) {
            const int q = o + lane;
            int vx = 0, vy = 0, vi = 0;
            if (q < n2) { vx = sx[src + q]; vy = sy[src + q]; vi = si[src + q]; }
            __syncwarp();
            if (q < n2) { sx[dst + q] = vx; sy[dst + q] = vy; si[dst + q] = vi; }
            __syncwarp();
          }
          if (lane == 0) s_cnt[ka] = is + 1 + n2;
        }
        __syncthreads();
      }
      // Output: lower chain, then the upper chain reversed.
      const int hl = s_cnt[0], hu = s_cnt[n0], ub = s_start[n0];
      const long long h = (long long)hl + (long long)hu - 2;
      if (threadIdx.x == 0) {
        plan->h = (u32)h; plan->h_lo = (u32)hl; plan->h_up = (u32)hu;
        if (h > cap) flag_error(plan, ERR_CAPACITY);
      }
      if (h > cap) return;
      for (int q = threadIdx.x; q < (int)h; q += K5_BLOCK)
        out[q] = q < hl ? si[q] : si[ub + (hu - 2) - (q - hl)];
      return;
    }
  }

  // ---------------- phase B, general case: merge chunk chains across the grid
  int2* cur_xy = h0_xy; int* cur_idx = h0_idx; u32* cur_cnt = cnt0;
  int2* nxt_xy = h1_xy; int* nxt_idx = h1_idx; u32* nxt_cnt = cnt1;
  const u32 maxchunks = max(cs.nchunk[0], cs.nchunk[1]);
  const int gw = blockIdx.x * K5_WARPS + wid, nw = nblk * K5_WARPS;
  for (u32 step = 1; step < maxchunks; step <<= 1) {
    if (!grid_barrier(plan, spin, nblk)) return;
    // B1: one warp per pair of nodes (or a lone node carried over).
    const u32 np0 = (cs.nchunk[0] + 2 * step - 1) / (2 * step);
    const u32 np1 = (cs.nchunk[1] + 2 * step - 1) / (2 * step);
    for (u32 job = gw; job < np0 + np1; job += nw) {
      const int c = job < np0 ? 0 : 1;
      const u32 p = c == 0 ? job : job - np0;
      const int sgn = c == 0 ? 1 : -1;
      const u32 ca = 2 * p * step, cb = ca + step;
      const u32 gca = cs.slot0[c] / C + ca;
      const int alpha = (int)__ldcg(&cur_cnt[gca]);
      int is = alpha - 1, js = 0, beta = 0;
      if (cb < cs.nchunk[c]) {
        const u32 gcb = cs.slot0[c] / C + cb;
        beta = (int)__ldcg(&cur_cnt[gcb]);
        GlobalChain A{cur_xy + (size_t)gca * C}, B{cur_xy + (size_t)gcb * C};
        bridge(A, alpha, B, beta, sgn, is, js);
      }
      if (lane == 0) {
        jobs[job] = make_int4(is, js, beta, 0);
        nxt_cnt[gca] = (u32)(is + 1 + (beta - js));
      }
    }
    if (!grid_barrier(plan, spin, nblk)) return;
    // B2: gather every merged node into the other buffer.
    const u32 span = 2 * step * C;
    const u32 total_slots = (cs.nchunk[0] + cs.nchunk[1]) * C;
    for (u32 q = blockIdx.x * K5_BLOCK + threadIdx.x; q < total_slots; q += nblk * K5_BLOCK) {
      const int c = q < cs.slot0[1] ? 0 : 1;
      const u32 rel = q - cs.slot0[c];
      const u32 p = rel / span, o = rel % span;
      const u32 job = c == 0 ? p : np0 + p;
      const int4 jd = __ldcg(&jobs[job]);
      const u32 merged = (u32)(jd.x + 1 + (jd.z - jd.y));
      if (o >= merged) continue;
      const u32 abase = cs.slot0[c] + p * span;
      u32 src;
      if (o <= (u32)jd.x) src = abase + o;
      else src = abase + step * C + (u32)jd.y + (o - (u32)jd.x - 1);
      nxt_xy[q] = __ldcg(&cur_xy[src]);
      nxt_idx[q] = __ldcg(&cur_idx[src]);
    }
    int2* t0 = cur_xy; cur_xy = nxt_xy; nxt_xy = t0;
    int* t1 = cur_idx; cur_idx = nxt_idx; nxt_idx = t1;
    u32* t2 = cur_cnt; cur_cnt = nxt_cnt; nxt_cnt = t2;
  }
  if (!grid_barrier(plan, spin, nblk)) return;

  // ---------------- output: lower chain, then the upper chain reversed
  const u32 hl = __ldcg(&cur_cnt[0]);
  const u32 hu = __ldcg(&cur_cnt[cs.slot0[1] / C]);
  const long long h = (long long)hl + (long long)hu - 2;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    plan->h = (u32)h; plan->h_lo = hl; plan->h_up = hu;
    if (h > cap) flag_error(plan, ERR_CAPACITY);
  }
  if (h > cap) return;
  for (u32 q = blockIdx.x * K5_BLOCK + threadIdx.x; q < (u32)h; q += nblk * K5_BLOCK) {
    int v;
    if (q < hl) v = __ldcg(&cur_idx[q]);
    else v = __ldcg(&cur_idx[cs.slot0[1] + (hu - 2) - (q - hl)]);
    out[q] = v;
  }
}

}  // namespace

int k5_chunk() { return K5_CHUNK; }
int k5_min_chunk() { return K5_MIN_CHUNK; }
size_t k5_dyn_smem() { return (size_t)K5_SMEM_PTS * 3 * sizeof(int); }

cudaError_t k5_configure(int* max_blocks_per_sm) {
  cudaError_t e = cudaFuncSetAttribute(k5_final, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)k5_dyn_smem());
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(max_blocks_per_sm, k5_final, K5_BLOCK,
                                                       k5_dyn_smem());
}

cudaError_t launch_k5(const int2* lo_xy, const int* lo_idx, const int2* up_xy, const int* up_idx,
                      Plan* plan, int2* h0_xy, int* h0_idx, int2* h1_xy, int* h1_idx, u32* cnt0,
                      u32* cnt1, int4* jobs, int* out, long long cap, int grid, cudaStream_t st) {
  void* args[] = {(void*)&lo_xy, (void*)&lo_idx, (void*)&up_xy, (void*)&up_idx, (void*)&plan,
                  (void*)&h0_xy, (void*)&h0_idx, (void*)&h1_xy, (void*)&h1_idx, (void*)&cnt0,
                  (void*)&cnt1, (void*)&jobs, (void*)&out, (void*)&cap};
  return cudaLaunchCooperativeKernel((const void*)k5_final, dim3(grid), dim3(K5_BLOCK), args,
                                     k5_dyn_smem(), st);
}

}  // namespace gbh
