// Block-level pieces of the learned filter proposal, shared by the single
// hull kernels (K6 / K8) and the batched kernel:
//   block_features  64 features and 32 directional extremes of a strided
//                   sample (centre = float64 mean; 32 angular bins of point
//                   fractions and of maximum radius over the largest;
//                   u_j = (cos 2 pi j/32, sin 2 pi j/32), ties to the
//                   smaller index);
//   block_mlp       64 -> 128 -> 128 -> 32 with ReLU, FP16 weights, FP32
//                   accumulation;
//   learned_polygon the exact convex hull (int64) of the quadrilateral's
//                   corners and the extremes of the 8 highest scores (ties:
//                   lower j), kept only when it encloses more area.
#pragma once

#include <cuda_fp16.h>

#include "hull_internal.cuh"

namespace gbh {
namespace learned {

constexpr int NB = 32;
constexpr int D0 = 64, D1 = 128, D2 = 128, D3 = 32;
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + D1 * D0, OFF_W2 = OFF_B1 + D1, OFF_B2 = OFF_W2 + D2 * D1,
              OFF_W3 = OFF_B2 + D2, OFF_B3 = OFF_W3 + D3 * D2, N_PARAMS = OFF_B3 + D3;
static_assert(N_PARAMS == 28960, "parameter count");

struct FeatSmem {
  double sum[2][32];
  u32 cnt[NB];
  float maxr[NB];
  float best[NB][32];
  u32 bidx[NB][32];
};

struct MlpSmem {
  float x[D0];
  float h1[D1];
  float h2[D2];
  float z[D3];
};

// Features of the sample i_k = floor(k n / S), k < S, of the points P[0, n).
// Writes x[64] (shared), ext_xy[32][2] and ext_idx[32].  All threads call.
template <int BLOCK>
__device__ void block_features(const int2* __restrict__ P, u32 n, u32 S, FeatSmem& sm, float* x,
                               int* ext_xy, int* ext_idx) {
  static_assert(BLOCK <= 1024 && BLOCK >= NB, "block size");
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  constexpr int NW = BLOCK / 32;
  double sx = 0.0, sy = 0.0;
  for (u32 k = threadIdx.x; k < S; k += BLOCK) {
    const int2 p = P[(u32)(((unsigned long long)k * n) / S)];
    sx += p.x; sy += p.y;
  }
  #pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    sx += __shfl_xor_sync(0xFFFFFFFFu, sx, o);
    sy += __shfl_xor_sync(0xFFFFFFFFu, sy, o);
  }
  if (lane == 0) { sm.sum[0][wid] = sx; sm.sum[1][wid] = sy; }
  if (threadIdx.x < NB) { sm.cnt[threadIdx.x] = 0; sm.maxr[threadIdx.x] = 0.f; }
  __syncthreads();
  double cx = 0.0, cy = 0.0;
  for (int w = 0; w < NW; ++w) { cx += sm.sum[0][w]; cy += sm.sum[1][w]; }
  const float fcx = (float)(cx / (double)S), fcy = (float)(cy / (double)S);
  float best[NB];
  u32 bidx[NB];
  float ux[NB / 2], uy[NB / 2];
  #pragma unroll
  for (int j = 0; j < NB / 2; ++j) {
    float sn, cs;
    sincosf(6.283185307179586f * (float)j / (float)NB, &sn, &cs);
    ux[j] = cs; uy[j] = sn;
    best[j] = -INFINITY; best[j + NB / 2] = -INFINITY;
    bidx[j] = 0xFFFFFFFFu; bidx[j + NB / 2] = 0xFFFFFFFFu;
  }
  for (u32 k = threadIdx.x; k < S; k += BLOCK) {
    const u32 i = (u32)(((unsigned long long)k * n) / S);
    const int2 p = P[i];
    const float dx = (float)p.x - fcx, dy = (float)p.y - fcy;
    const float ang = atan2f(dy, dx);
    int b = (int)floorf((ang + 3.14159265358979f) * ((float)NB / 6.283185307179586f));
    b = b < 0 ? 0 : (b >= NB ? NB - 1 : b);
    atomicAdd(&sm.cnt[b], 1u);
    atomicMax(reinterpret_cast<int*>(&sm.maxr[b]), __float_as_int(sqrtf(dx * dx + dy * dy)));
    const float fx = (float)p.x, fy = (float)p.y;
    #pragma unroll
    for (int j = 0; j < NB / 2; ++j) {
      const float d = ux[j] * fx + uy[j] * fy;
      if (d > best[j]) { best[j] = d; bidx[j] = i; }
      if (-d > best[j + NB / 2]) { best[j + NB / 2] = -d; bidx[j + NB / 2] = i; }
    }
  }
  #pragma unroll
  for (int j = 0; j < NB; ++j) {
    float v = best[j];
    u32 ix = bidx[j];
    #pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float v2 = __shfl_xor_sync(0xFFFFFFFFu, v, o);
      const u32 i2 = __shfl_xor_sync(0xFFFFFFFFu, ix, o);
      if (v2 > v || (v2 == v && i2 < ix)) { v = v2; ix = i2; }
    }
    if (lane == 0) { sm.best[j][wid] = v; sm.bidx[j][wid] = ix; }
  }
  __syncthreads();
  if (threadIdx.x < NB) {
    const int j = threadIdx.x;
    float v = -INFINITY;
    u32 ix = 0xFFFFFFFFu;
    for (int w = 0; w < NW; ++w) {
      const float v2 = sm.best[j][w];
      const u32 i2 = sm.bidx[j][w];
      if (v2 > v || (v2 == v && i2 < ix)) { v = v2; ix = i2; }
    }
    ext_idx[j] = (int)ix;
    const int2 p = P[ix];
    ext_xy[2 * j] = p.x;
    ext_xy[2 * j + 1] = p.y;
    float mr = 0.f;
    for (int q = 0; q < NB; ++q) mr = fmaxf(mr, sm.maxr[q]);
    x[j] = (float)sm.cnt[j] / (float)S;
    x[NB + j] = mr > 0.f ? sm.maxr[j] / mr : 0.f;
  }
  __syncthreads();
}

// MLP on sm.x into sm.z; needs at least 128 threads, all threads call.
__device__ __forceinline__ void block_mlp(const __half* __restrict__ w16, MlpSmem& sm) {
  const int t = threadIdx.x;
  if (t < D1) {
    float a = __half2float(w16[OFF_B1 + t]);
    for (int k = 0; k < D0; ++k) a = fmaf(__half2float(w16[OFF_W1 + t * D0 + k]), sm.x[k], a);
    sm.h1[t] = fmaxf(a, 0.f);
  }
  __syncthreads();
  if (t < D2) {
    float a = __half2float(w16[OFF_B2 + t]);
    for (int k = 0; k < D1; ++k) a = fmaf(__half2float(w16[OFF_W2 + t * D1 + k]), sm.h1[k], a);
    sm.h2[t] = fmaxf(a, 0.f);
  }
  __syncthreads();
  if (t < D3) {
    float a = __half2float(w16[OFF_B3 + t]);
    for (int k = 0; k < D2; ++k) a = fmaf(__half2float(w16[OFF_W3 + t * D2 + k]), sm.h2[k], a);
    sm.z[t] = a;
  }
  __syncthreads();
}

__device__ __forceinline__ long long orient64(int ax, int ay, int bx, int by, int cx, int cy) {
  return (long long)(bx - ax) * (cy - ay) - (long long)(by - ay) * (cx - ax);
}

// Exact convex hull (strict vertices, CCW from the lexicographic minimum)
// of m <= 16 points (px/py reordered in place; hx/hy need 2m + 1 slots);
// single thread.  Returns the vertex count.
__device__ inline int small_hull(int* px, int* py, int m, int* hx, int* hy) {
  for (int i = 1; i < m; ++i) {
    const int x = px[i], y = py[i];
    int j = i - 1;
    while (j >= 0 && (px[j] > x || (px[j] == x && py[j] > y))) { px[j + 1] = px[j]; py[j + 1] = py[j]; --j; }
    px[j + 1] = x; py[j + 1] = y;
  }
  int u = 0;
  for (int i = 0; i < m; ++i)
    if (u == 0 || px[u - 1] != px[i] || py[u - 1] != py[i]) { px[u] = px[i]; py[u] = py[i]; ++u; }
  if (u <= 2) {
    for (int i = 0; i < u; ++i) { hx[i] = px[i]; hy[i] = py[i]; }
    return u;
  }
  int k = 0;
  for (int i = 0; i < u; ++i) {
    while (k >= 2 && orient64(hx[k - 2], hy[k - 2], hx[k - 1], hy[k - 1], px[i], py[i]) <= 0) --k;
    hx[k] = px[i]; hy[k] = py[i]; ++k;
  }
  const int lower = k + 1;
  for (int i = u - 2; i >= 0; --i) {
    while (k >= lower && orient64(hx[k - 2], hy[k - 2], hx[k - 1], hy[k - 1], px[i], py[i]) <= 0) --k;
    hx[k] = px[i]; hy[k] = py[i]; ++k;
  }
  return k - 1;
}

// Twice the area (shoelace, exact int64 for |coordinates| <= 2^29).
__device__ inline long long area2(const int* hx, const int* hy, int k) {
  long long a = 0;
  for (int i = 0; i < k; ++i) {
    const int j = (i + 1) % k;
    a += (long long)hx[i] * hy[j] - (long long)hx[j] * hy[i];
  }
  return a;
}

// Single thread: the learned polygon from the scores z, the extremes and
// the quadrilateral (qx, qy, nq).  Returns its corner count (written to
// outx / outy, <= kMaxCorners), or 0 when the quadrilateral is kept.
__device__ inline int learned_polygon(const float* z, const int* ext_xy, const int* qx, const int* qy,
                                      int nq, int* outx, int* outy) {
  bool used[D3];
  for (int j = 0; j < D3; ++j) used[j] = false;
  int px[16], py[16], m = 0;
  for (int j = 0; j < nq && j < 4; ++j) { px[m] = qx[j]; py[m] = qy[j]; ++m; }
  for (int pick = 0; pick < 8; ++pick) {
    int bj = -1;
    float bv = -INFINITY;
    for (int j = 0; j < D3; ++j)
      if (!used[j] && (bj < 0 || z[j] > bv)) { bv = z[j]; bj = j; }
    used[bj] = true;
    px[m] = ext_xy[2 * bj]; py[m] = ext_xy[2 * bj + 1]; ++m;
  }
  int hx[34], hy[34];
  const int k = small_hull(px, py, m, hx, hy);
  const long long aq = nq >= 3 ? area2(qx, qy, nq) : 0;
  if (k < 3 || k > kMaxCorners || area2(hx, hy, k) <= aq) return 0;
  for (int j = 0; j < k; ++j) { outx[j] = hx[j]; outy[j] = hy[j]; }
  return k;
}

}  // namespace learned
}  // namespace gbh
