// K1: the four extreme points (Section 2.1 step 1, Section 3.1).
//
// One streaming pass over the int32 (x, y) pairs with 128-bit loads (two
// points per load).  Each candidate is a 64-bit lexicographic key plus the
// input index; all four extremes are minima of (key, idx):
//   P_minx: key (x, y)        P_maxx: complement of key (x, y)
//   P_miny: key (y, x)        P_maxy: complement of key (y, x)
// so ties resolve lexicographically and then to the smallest index.
// With a sample buffer it also copies every kSampleStride-th point there
// (sample[i] = point i kSampleStride), the input of the fused front's
// witnesses, while the points are in registers anyway.
// Warp shuffles, then a block reduction, then the last block to finish
// reduces the per-block partials and builds the Plan: the range check, the
// counter-clockwise filter polygon, the radix-key layout, the epoch, and
// zeroed counters and histograms for the kernels that follow.
#include "hull_internal.cuh"
#include "kernels.h"

namespace gbh {

namespace {

__device__ __forceinline__ u32 ord(int v) { return (u32)v ^ 0x80000000u; }

struct Best {
  u64 k[4];
  u32 i[4];
  // Current x of P_minx / P_maxx and y of P_miny / P_maxy candidates: a
  // point strictly inside this box cannot change any extreme.
  int bx0, bx1, by0, by1;
};

__device__ __forceinline__ void best_init(Best& b) {
  #pragma unroll
  for (int j = 0; j < 4; ++j) { b.k[j] = ~0ull; b.i[j] = 0xFFFFFFFFu; }
  b.bx0 = 0x7FFFFFFF; b.bx1 = (int)0x80000000; b.by0 = 0x7FFFFFFF; b.by1 = (int)0x80000000;
}

__device__ __forceinline__ bool lt_ki(u64 ka, u32 ia, u64 kb, u32 ib) {
  return ka < kb || (ka == kb && ia < ib);
}

// Points reach a thread in increasing index order, so a strict key
// comparison keeps the smallest index among equal keys.
__device__ __forceinline__ void consider(Best& b, int x, int y, u32 idx) {
  if (x > b.bx0 && x < b.bx1 && y > b.by0 && y < b.by1) return;
  u32 ox = ord(x), oy = ord(y);
  u64 kxy = ((u64)ox << 32) | oy;
  u64 kyx = ((u64)oy << 32) | ox;
  if (kxy < b.k[0]) { b.k[0] = kxy; b.i[0] = idx; b.bx0 = min(b.bx0, x); }
  if (~kxy < b.k[1]) { b.k[1] = ~kxy; b.i[1] = idx; b.bx1 = max(b.bx1, x); }
  if (kyx < b.k[2]) { b.k[2] = kyx; b.i[2] = idx; b.by0 = min(b.by0, y); }
  if (~kyx < b.k[3]) { b.k[3] = ~kyx; b.i[3] = idx; b.by1 = max(b.by1, y); }
}

// Two points at once: a single warp vote skips both when every lane's
// points lie strictly inside that lane's current box (the common case).
__device__ __forceinline__ void consider2(Best& b, int4 v, u32 idx) {
  const bool out = !(v.x > b.bx0 && v.x < b.bx1 && v.y > b.by0 && v.y < b.by1) ||
                   !(v.z > b.bx0 && v.z < b.bx1 && v.w > b.by0 && v.w < b.by1);
  if (__any_sync(__activemask(), out)) {
    consider(b, v.x, v.y, idx);
    consider(b, v.z, v.w, idx + 1);
  }
}

__device__ __forceinline__ void merge_best(Best& a, const u64* k, const u32* i) {
  #pragma unroll
  for (int j = 0; j < 4; ++j)
    if (lt_ki(k[j], i[j], a.k[j], a.i[j])) { a.k[j] = k[j]; a.i[j] = i[j]; }
}

__device__ __forceinline__ void warp_reduce(Best& b) {
  #pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    u64 k[4];
    u32 i[4];
    #pragma unroll
    for (int j = 0; j < 4; ++j) {
      k[j] = __shfl_xor_sync(0xFFFFFFFFu, b.k[j], o);
      i[j] = __shfl_xor_sync(0xFFFFFFFFu, b.i[j], o);
    }
    merge_best(b, k, i);
  }
}

__device__ __forceinline__ u32 bitlen(u32 v) { return v ? 32u - (u32)__clz(v) : 0u; }

// Builds the Plan from the final extremes (single thread).
__device__ void finish_plan(Plan* plan, const Best& b) {
  int ex[4], ey[4];
  ex[0] = (int)(u32)((b.k[0] >> 32) ^ 0x80000000u);  ey[0] = (int)((u32)b.k[0] ^ 0x80000000u);
  u64 k1 = ~b.k[1];
  ex[1] = (int)(u32)((k1 >> 32) ^ 0x80000000u);      ey[1] = (int)((u32)k1 ^ 0x80000000u);
  ey[2] = (int)(u32)((b.k[2] >> 32) ^ 0x80000000u);  ex[2] = (int)((u32)b.k[2] ^ 0x80000000u);
  u64 k3 = ~b.k[3];
  ey[3] = (int)(u32)((k3 >> 32) ^ 0x80000000u);      ex[3] = (int)((u32)k3 ^ 0x80000000u);
  for (int j = 0; j < 4; ++j) { plan->ext_idx[j] = (int)b.i[j]; plan->ext_x[j] = ex[j]; plan->ext_y[j] = ey[j]; }

  // The bounding box is spanned by the extremes, so the range check needs
  // no per-point work.
  // Starts the call's error word afresh.
  bool bad = ex[0] < -kCoordLimit || ex[1] > kCoordLimit || ey[2] < -kCoordLimit || ey[3] > kCoordLimit;
  plan->error = bad ? ERR_RANGE : 0u;

  // Filter polygon: P_minx, P_miny, P_maxx, P_maxy (counter-clockwise along
  // the hull), cyclically repeated corners removed.
  const int order[4] = {0, 2, 1, 3};
  int k = 0;
  int cx[4], cy[4];
  for (int j = 0; j < 4; ++j) {
    int x = ex[order[j]], y = ey[order[j]];
    if (k > 0 && cx[k - 1] == x && cy[k - 1] == y) continue;
    cx[k] = x; cy[k] = y; ++k;
  }
  while (k > 1 && cx[k - 1] == cx[0] && cy[k - 1] == cy[0]) --k;
  plan->ncorner = k;
  for (int j = 0; j < k; ++j) { plan->cx[j] = cx[j]; plan->cy[j] = cy[j]; }

  // Radix key: ((x - x0) << ybits) | (y - y0), order-isomorphic to the
  // lexicographic (x, y) order; only the bits that vary are sorted.
  plan->key_x0 = ex[0];
  plan->key_y0 = ey[2];
  u32 xr = (u32)(ex[1] - ex[0]);
  u32 yr = (u32)(ey[3] - ey[2]);
  u32 yb = bitlen(yr), xb = bitlen(xr);
  plan->ybits = yb;
  plan->kbits = xb + yb;
  plan->npasses = (xb + yb + kRadixBits - 1) / kRadixBits;
  plan->sorted_in_b = plan->npasses & 1u;
  plan->fshift = xb + yb > (u32)kBinBits ? xb + yb - (u32)kBinBits : 0u;
  plan->ngroups = 0;
}

// Warp, block and grid reduction of the extremes; the last block to finish
// reduces the per-block partials and builds the Plan.
template <int BLOCK>
__device__ void k1_reduce_finish(Best& b, u32 n, u32 spin_limit, Plan* plan, ExtPartial* __restrict__ partials,
                                 const u32* raw_count = nullptr) {
  warp_reduce(b);

  constexpr int NW = BLOCK / 32;
  __shared__ u64 sk[NW][4];
  __shared__ u32 si[NW][4];
  __shared__ bool am_last;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0)
    for (int q = 0; q < 4; ++q) { sk[wid][q] = b.k[q]; si[wid][q] = b.i[q]; }
  __syncthreads();
  if (wid == 0) {
    best_init(b);
    if (lane < NW) {
      u64 k[4]; u32 i[4];
      for (int q = 0; q < 4; ++q) { k[q] = sk[lane][q]; i[q] = si[lane][q]; }
      merge_best(b, k, i);
    }
    warp_reduce(b);
    if (lane == 0) {
      ExtPartial* P = &partials[blockIdx.x];
      for (int q = 0; q < 4; ++q) { P->key[q] = b.k[q]; P->idx[q] = b.i[q]; }
      __threadfence();
      u32 t = atomicAdd(&plan->k1_done, 1u);
      am_last = (t == gridDim.x - 1);
    }
  }
  __syncthreads();
  if (!am_last) return;

  // Last block: reduce all partials and build the Plan.
  __threadfence();
  best_init(b);
  for (u32 p = threadIdx.x; p < gridDim.x; p += BLOCK) {
    const volatile ExtPartial* P = &partials[p];
    u64 k[4]; u32 i[4];
    for (int q = 0; q < 4; ++q) { k[q] = P->key[q]; i[q] = P->idx[q]; }
    merge_best(b, k, i);
  }
  warp_reduce(b);
  if (lane == 0)
    for (int q = 0; q < 4; ++q) { sk[wid][q] = b.k[q]; si[wid][q] = b.i[q]; }
  __syncthreads();
  // Zero the per-call counters and histograms for the later kernels.
  for (int q = threadIdx.x; q < kMaxPasses * kRadix; q += BLOCK) (&plan->hist[0][0])[q] = 0u;
  for (int q = threadIdx.x; q < kNumCounters; q += BLOCK) plan->ctr[q] = 0u;
  if (threadIdx.x == 0) {
    best_init(b);
    for (int w = 0; w < NW; ++w) merge_best(b, sk[w], si[w]);
    plan->n = n;
    plan->spin_limit = spin_limit;
    finish_plan(plan, b);
    plan->epoch += kEpochStride;
    plan->s = 0; plan->s_quad = 0; plan->r_lo = 0; plan->r_up = 0; plan->h = 0; plan->h_lo = 0; plan->h_up = 0;
    plan->s_raw = raw_count ? ld_volatile_u32(raw_count) : 0u;
    plan->learned_used = 0;
    plan->k1_done = 0;
  }
}

template <int BLOCK, bool VEC>
__global__ void __launch_bounds__(BLOCK)
k1_extremes(const int* __restrict__ xy, u32 n, u32 spin_limit, Plan* plan,
            ExtPartial* __restrict__ partials, int2* __restrict__ sample) {
  constexpr u32 kPairStride = kSampleStride / 2;   // pair j holds sample point j / kPairStride
  static_assert(kSampleStride % 2 == 0, "sampled points start a pair");
  Best b;
  best_init(b);
  const u32 tid = blockIdx.x * BLOCK + threadIdx.x;
  const u32 nthreads = gridDim.x * BLOCK;
  // Every thread's skip box starts as the bounding box of points the block
  // has read: a point strictly inside a box spanned by input points cannot
  // be an extreme.  (The points that span it still reach their owners as
  // candidates: they lie on or outside that box.)  With 16-byte alignment
  // the box comes from the block's first round of loads (8 int4 per thread,
  // 16 * BLOCK points, read anyway); otherwise from a strided sample of
  // BLOCK points.  A box from thousands of points leaves few points outside
  // it, and a warp whose points all lie inside skips them with one vote.
  __shared__ int s_box[4];
  if (threadIdx.x == 0) { s_box[0] = 0x7FFFFFFF; s_box[1] = (int)0x80000000; s_box[2] = 0x7FFFFFFF; s_box[3] = (int)0x80000000; }
  __syncthreads();
  auto seed_box = [&](int x0, int x1, int y0, int y1) {
    #pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      x0 = min(x0, __shfl_xor_sync(0xFFFFFFFFu, x0, o));
      x1 = max(x1, __shfl_xor_sync(0xFFFFFFFFu, x1, o));
      y0 = min(y0, __shfl_xor_sync(0xFFFFFFFFu, y0, o));
      y1 = max(y1, __shfl_xor_sync(0xFFFFFFFFu, y1, o));
    }
    if ((threadIdx.x & 31) == 0) {
      atomicMin(&s_box[0], x0); atomicMax(&s_box[1], x1);
      atomicMin(&s_box[2], y0); atomicMax(&s_box[3], y1);
    }
    __syncthreads();
    b.bx0 = s_box[0]; b.bx1 = s_box[1]; b.by0 = s_box[2]; b.by1 = s_box[3];
  };
  if (VEC) {
    // 16-byte aligned: pair j holds points 2j and 2j + 1.
    const int4* p4 = reinterpret_cast<const int4*>(xy);
    const u32 npair = n >> 1;
    u32 j = tid;
    int4 v[8];
    const bool first = j + 7 * nthreads < npair;
    {
      int x0 = 0x7FFFFFFF, x1 = (int)0x80000000, y0 = 0x7FFFFFFF, y1 = (int)0x80000000;
      if (first) {
        #pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = p4[j + u * nthreads];
        #pragma unroll
        for (int u = 0; u < 8; ++u) {
          x0 = min(x0, min(v[u].x, v[u].z)); x1 = max(x1, max(v[u].x, v[u].z));
          y0 = min(y0, min(v[u].y, v[u].w)); y1 = max(y1, max(v[u].y, v[u].w));
        }
      }
      seed_box(x0, x1, y0, y1);
    }
    auto take8 = [&](u32 jj) {
      #pragma unroll
      for (int u = 0; u < 8; ++u) consider2(b, v[u], 2 * (jj + u * nthreads));
      if (sample) {
        #pragma unroll
        for (int u = 0; u < 8; ++u)
          if ((jj + u * nthreads) % kPairStride == 0) sample[(jj + u * nthreads) / kPairStride] = make_int2(v[u].x, v[u].y);
      }
    };
    if (first) {
      take8(j);
      j += 8 * nthreads;
    }
    for (; j + 7 * nthreads < npair; j += 8 * nthreads) {
      #pragma unroll
      for (int u = 0; u < 8; ++u) v[u] = p4[j + u * nthreads];
      take8(j);
    }
    for (; j < npair; j += nthreads) {
      int4 w = p4[j];
      consider(b, w.x, w.y, 2 * j);
      consider(b, w.z, w.w, 2 * j + 1);
      if (sample && j % kPairStride == 0) sample[j / kPairStride] = make_int2(w.x, w.y);
    }
    if ((n & 1u) && tid == 0) {
      consider(b, xy[2 * (n - 1)], xy[2 * (n - 1) + 1], n - 1);
      if (sample && (n - 1) % kSampleStride == 0) sample[(n - 1) / kSampleStride] = make_int2(xy[2 * (n - 1)], xy[2 * (n - 1) + 1]);
    }
  } else {
    const int2* p2 = reinterpret_cast<const int2*>(xy);
    {
      const u32 step = n / BLOCK + 1;
      const u32 jj = threadIdx.x * step;
      int x0 = 0x7FFFFFFF, x1 = (int)0x80000000, y0 = 0x7FFFFFFF, y1 = (int)0x80000000;
      if (jj < n) { const int2 q = p2[jj]; x0 = x1 = q.x; y0 = y1 = q.y; }
      seed_box(x0, x1, y0, y1);
    }
    for (u32 j = tid; j < n; j += nthreads) {
      int2 v = p2[j];
      consider(b, v.x, v.y, j);
      if (sample && j % kSampleStride == 0) sample[j / kSampleStride] = v;
    }
  }
  k1_reduce_finish<BLOCK>(b, n, spin_limit, plan, partials);
}

// ---- K1 of the single-read front: the extremes and the sample polygon's
// filter in one pass.  A point strictly inside the sample polygon (PolyTab,
// k0_poly.cu: xl < x < xr and strictly inside its slab's y interval) is
// strictly inside the hull, so it is neither an extreme nor a vertex: it is
// dropped.  Every other point is a candidate for the
// extremes and is staged in its warp's slice of shared memory; a warp
// flushes its slice with one atomic reservation into (rxy, ridx), in no
// particular order (the later kernels order the survivors themselves).
// Each warp streams one contiguous run of 8 x 32 pairs per round (16-byte
// aligned input); the rest, and an odd last point, go one pair per lane.
constexpr int K1P_BLOCK = 512;
constexpr int K1P_WARPS = K1P_BLOCK / 32;
constexpr int K1P_SLICE = 256;                 // staged points per warp (a half round: 32 x 8)

struct K1PSmem {
  int2 sxy[K1P_WARPS][K1P_SLICE];
  u32 sidx[K1P_WARPS][K1P_SLICE];
  int2 yb[kPolySlabs];
};

__global__ void __launch_bounds__(K1P_BLOCK, 2)
k1_poly(const int* __restrict__ xy, u32 n, u32 spin_limit, Plan* plan, ExtPartial* __restrict__ partials,
        const PolyTab* __restrict__ T, u32* raw_count, int2* __restrict__ rxy, u32* __restrict__ ridx) {
  extern __shared__ __align__(16) unsigned char k1p_smem[];
  K1PSmem& S = *reinterpret_cast<K1PSmem*>(k1p_smem);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const u32 lt = (1u << lane) - 1u;
  const int ok = T->ok;
  const int xl = T->xl, xr = T->xr;
  const u32 sh = T->sh;

  if (ok) {
    const u32 nslab = T->nslab;
    for (u32 q = threadIdx.x; q < nslab; q += K1P_BLOCK) S.yb[q] = T->yb[q];
  }
  __syncthreads();
  // Branch-free: every lane looks its slab up (slab 0 when x is outside the
  // range, whose answer is then ignored), so a warp never splits here.
  auto inside = [&](int x, int y) -> bool {
    const bool inx = ok && x > xl && x < xr;
    const int2 q = S.yb[inx ? (u32)(x - xl) >> sh : 0u];
    return inx & (y > q.x) & (y < q.y);
  };
  Best b;
  best_init(b);
  int2* sxy = S.sxy[wid];
  u32* sidx = S.sidx[wid];
  u32 fill = 0;                                   // uniform over the warp
  auto flush = [&]() {
    __syncwarp();
    u32 base = 0;
    if (lane == 0) base = atomicAdd(raw_count, fill);
    base = __shfl_sync(0xFFFFFFFFu, base, 0);
    for (u32 q = lane; q < fill; q += 32) {
      if (base + q < n) { rxy[base + q] = sxy[q]; ridx[base + q] = sidx[q]; }
      else flag_error(plan, ERR_INTERNAL);
    }
    __syncwarp();
    fill = 0;
  };
  // Up to 8 points per lane (validity in `valid`): the survivors become
  // extreme candidates and are staged (the whole warp calls it).
  auto take = [&](const int* px, const int* py, const u32* pi, u32 valid, int cntpts) {
    u32 keep = 0;
    for (int e = 0; e < cntpts; ++e)
      if (((valid >> e) & 1u) && !inside(px[e], py[e])) keep |= 1u << e;
    if (!__any_sync(0xFFFFFFFFu, keep != 0)) return;
    for (int e = 0; e < cntpts; ++e)
      if ((keep >> e) & 1u) consider(b, px[e], py[e], pi[e]);
    const u32 cnt = __popc(keep);
    u32 inc = cnt;
    #pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const u32 t = __shfl_up_sync(0xFFFFFFFFu, inc, o);
      if (lane >= o) inc += t;
    }
    const u32 tot = __shfl_sync(0xFFFFFFFFu, inc, 31);
    if (fill + tot > (u32)K1P_SLICE) flush();
    u32 pos = fill + inc - cnt;
    for (int e = 0; e < cntpts; ++e)
      if ((keep >> e) & 1u) { sxy[pos] = make_int2(px[e], py[e]); sidx[pos] = pi[e]; ++pos; }
    fill += tot;
  };
  const int4* p4 = reinterpret_cast<const int4*>(xy);
  const u32 npair = n >> 1;
  const u32 nthreads = gridDim.x * K1P_BLOCK;
  const u32 gw = (blockIdx.x * K1P_BLOCK + threadIdx.x) >> 5, nwarps = nthreads >> 5;
  u32 R = 0;
  for (; R + 8u * nthreads <= npair; R += 8u * nthreads) {
    const u32 u0 = R + gw * 256u + lane;
    int4 v[8];
    #pragma unroll
    for (int u = 0; u < 8; ++u) v[u] = p4[u0 + 32u * u];
    #pragma unroll
    for (int h = 0; h < 2; ++h) {
      int px[8], py[8];
      u32 pi[8];
      #pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int4 w = v[4 * h + q];
        const u32 j = u0 + 32u * (4 * h + q);
        px[2 * q] = w.x; py[2 * q] = w.y; pi[2 * q] = 2u * j;
        px[2 * q + 1] = w.z; py[2 * q + 1] = w.w; pi[2 * q + 1] = 2u * j + 1u;
      }
      take(px, py, pi, 0xFFu, 8);
    }
  }
  // The rest of the pairs, one per lane; then the odd last point.
  for (u32 wb = R + gw * 32u; wb < npair; wb += nwarps * 32u) {
    const u32 j = wb + lane;
    int px[2] = {0, 0}, py[2] = {0, 0};
    u32 pi[2] = {2u * j, 2u * j + 1u};
    u32 valid = 0;
    if (j < npair) {
      const int4 w = p4[j];
      px[0] = w.x; py[0] = w.y; px[1] = w.z; py[1] = w.w;
      valid = 3u;
    }
    take(px, py, pi, valid, 2);
  }
  if ((n & 1u) && gw == 0) {
    int px[1] = {0}, py[1] = {0};
    u32 pi[1] = {n - 1};
    u32 valid = 0;
    if (lane == 0) {
      px[0] = xy[2 * (n - 1)]; py[0] = xy[2 * (n - 1) + 1]; valid = 1u;
    }
    take(px, py, pi, valid, 1);
  }
  if (fill) flush();
  __threadfence();
  k1_reduce_finish<K1P_BLOCK>(b, n, spin_limit, plan, partials, raw_count);
}

}  // namespace

static int g_k1_occ = 0;

// Enough blocks to cover the input, but never more than fit on the GPU at
// once (a partial second wave would idle most SMs).
int k1_grid(u32 n, int num_sms) {
  const int block = 512;
  if (g_k1_occ == 0) {
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k1_extremes<512, true>, block, 0) != cudaSuccess || occ < 1)
      occ = 1;
    g_k1_occ = occ;
  }
  long long want = ((long long)(n / 2) + block * 8 - 1) / (block * 8);
  long long cap = (long long)num_sms * g_k1_occ;
  if (want < 1) want = 1;
  return (int)(want < cap ? want : cap);
}

cudaError_t launch_k1(const int* xy, u32 n, u32 spin_limit, Plan* plan, ExtPartial* partials,
                      int grid, cudaStream_t st, int2* sample) {
  const bool vec = (reinterpret_cast<uintptr_t>(xy) & 15u) == 0;
  if (vec)
    k1_extremes<512, true><<<grid, 512, 0, st>>>(xy, n, spin_limit, plan, partials, sample);
  else
    k1_extremes<512, false><<<grid, 512, 0, st>>>(xy, n, spin_limit, plan, partials, sample);
  return cudaGetLastError();
}


cudaError_t k1_poly_configure() {
  return cudaFuncSetAttribute(k1_poly, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(K1PSmem));
}

cudaError_t launch_k1_poly(const int* xy, u32 n, u32 spin_limit, Plan* plan, ExtPartial* partials, const PolyTab* T,
                           u32* raw_count, int2* rxy, u32* ridx, int num_sms, cudaStream_t st) {
  k1_poly<<<num_sms * 2, K1P_BLOCK, sizeof(K1PSmem), st>>>(xy, n, spin_limit, plan, partials, T, raw_count, rxy, ridx);
  return cudaGetLastError();
}

}  // namespace gbh
