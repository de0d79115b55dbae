// Learned filter proposal (the project's addition beside the paper's
// quadrilateral of Section 2.1 step 2 / Section 3.1):
//
//   K6  features of a strided sample of the input: its centre, a 32-bin
//       angular histogram (fraction of points, maximum radius normalised by
//       the largest) = 64 features, and the sample's extreme point in each
//       of 32 directions u_j = (cos 2 pi j / 32, sin 2 pi j / 32);
//   K8  inference of an MLP 64 -> 128 -> 128 -> 32 (ReLU, FP16 weights,
//       FP32 accumulation); the 8 highest scores pick 8 directions, and the
//       filter polygon becomes the exact (int64) convex hull of the four
//       quadrilateral corners and those 8 extremes (at most 12 corners).  It
//       contains the quadrilateral, so it never discards less; points are
//       discarded only when strictly inside a polygon spanned by input
//       points, so the hull stays exact whatever the weights;
//   K10 labels for training: for every direction j the discard fraction of
//       hull(quad corners + e_j) minus the quadrilateral's, counted exactly;
//   training: batched forward / backward of the MLP (FP32 FFMA tiles, the
//       forward pass on the FP16-rounded weights used at inference), mean
//       squared error on the labels, Adam on FP32 master weights.
#include <cmath>

#include "hull_internal.cuh"
#include "kernels.h"
#include "learned_common.cuh"

namespace gbh {

using namespace learned;

namespace {

constexpr int F_SAMPLE = 16384;
constexpr int F_BLOCK = 512;

__device__ __forceinline__ float fp16r(float w) { return __half2float(__float2half_rn(w)); }

// K6: features and extremes of the sample of one input (one block).
__global__ void __launch_bounds__(F_BLOCK)
k6_features(const int* __restrict__ xy, u32 n, float* __restrict__ feat, int* __restrict__ ext,
            int* __restrict__ ext_xy) {
  __shared__ FeatSmem sm;
  __shared__ float s_x[D0];
  const u32 S = n < (u32)F_SAMPLE ? n : (u32)F_SAMPLE;
  block_features<F_BLOCK>(reinterpret_cast<const int2*>(xy), n, S, sm, s_x, ext_xy, ext);
  if (threadIdx.x < D0) feat[threadIdx.x] = s_x[threadIdx.x];
}

// K8: inference on one feature vector and the filter polygon (one block).
__global__ void __launch_bounds__(128)
k8_infer(const float* __restrict__ feat, const __half* __restrict__ w16, const int* __restrict__ ext_xy,
         Plan* plan) {
  __shared__ MlpSmem sm;
  if (plan->error & ERR_RANGE) return;
  if (threadIdx.x < D0) sm.x[threadIdx.x] = feat[threadIdx.x];
  __syncthreads();
  block_mlp(w16, sm);
  if (threadIdx.x != 0) return;
  int qx[4], qy[4], ox[kMaxCorners], oy[kMaxCorners];
  const int nq = plan->ncorner < 4 ? plan->ncorner : 4;
  for (int j = 0; j < nq; ++j) { qx[j] = plan->cx[j]; qy[j] = plan->cy[j]; }
  const int k = learned_polygon(sm.z, ext_xy, qx, qy, nq, ox, oy);
  if (k > 0) {
    plan->ncorner = k;
    for (int j = 0; j < k; ++j) { plan->cx[j] = ox[j]; plan->cy[j] = oy[j]; }
    plan->learned_used = 1;
  }
}

// K6 + K8 in one launch behind a gate (the pipeline's path): the
// quadrilateral's discard on PG_SAMPLE strided points i_k = floor(k n / G)
// first; when it discards PG_DISCARD of them or more, there is too little
// left for a larger polygon to discard and the quadrilateral stays (no
// features, no inference: the call costs this one short launch).
// Otherwise the features, the MLP and the polygon exactly as K6 and K8.
constexpr int PG_SAMPLE = F_BLOCK;
constexpr float PG_DISCARD = 0.95f;

__global__ void __launch_bounds__(F_BLOCK)
k6_propose(const int* __restrict__ xy, u32 n, const __half* __restrict__ w16, float* __restrict__ feat,
           int* __restrict__ ext, int* __restrict__ ext_xy, Plan* plan) {
  __shared__ FeatSmem sm;
  __shared__ MlpSmem msm;
  __shared__ u32 s_in;
  if (plan->error & ERR_RANGE) return;
  const int2* P = reinterpret_cast<const int2*>(xy);
  const int k = plan->ncorner < 4 ? plan->ncorner : 4;
  if (threadIdx.x == 0) s_in = 0;
  __syncthreads();
  const u32 G = n < (u32)PG_SAMPLE ? n : (u32)PG_SAMPLE;
  if (threadIdx.x < G && k >= 3) {
    const int2 p = P[(u32)(((unsigned long long)threadIdx.x * n) / G)];
    bool in = true;
    for (int j = 0; j < k && in; ++j) {
      const int jn = j + 1 < k ? j + 1 : 0;
      in = orient(plan->cx[j], plan->cy[j], plan->cx[jn], plan->cy[jn], p.x, p.y) > 0;
    }
    if (in) atomicAdd(&s_in, 1u);
  }
  __syncthreads();
  if ((float)s_in >= PG_DISCARD * (float)G) return;
  const u32 S = n < (u32)F_SAMPLE ? n : (u32)F_SAMPLE;
  block_features<F_BLOCK>(P, n, S, sm, msm.x, ext_xy, ext);
  if (threadIdx.x < D0) feat[threadIdx.x] = msm.x[threadIdx.x];
  __syncthreads();
  block_mlp(w16, msm);
  if (threadIdx.x != 0) return;
  int qx[4], qy[4], ox[kMaxCorners], oy[kMaxCorners];
  for (int j = 0; j < k; ++j) { qx[j] = plan->cx[j]; qy[j] = plan->cy[j]; }
  const int kk = learned_polygon(msm.z, ext_xy, qx, qy, k, ox, oy);
  if (kk > 0) {
    plan->ncorner = kk;
    for (int j = 0; j < kk; ++j) { plan->cx[j] = ox[j]; plan->cy[j] = oy[j]; }
    plan->learned_used = 1;
  }
}

// K10: exact counts of points strictly inside the quadrilateral (slot 32)
// and inside hull(quad corners + e_j) (slot j), for one instance.
__global__ void __launch_bounds__(256)
k10_labels(const int* __restrict__ xy, u32 n, const int* __restrict__ quad, int nq,
           const int* __restrict__ ext_xy, unsigned long long* __restrict__ counts) {
  __shared__ int s_px[NB + 1][8], s_py[NB + 1][8], s_k[NB + 1];
  __shared__ u32 s_c[NB + 1];
  if (threadIdx.x <= NB) {
    const int j = threadIdx.x;
    int px[8], py[8], m = 0;
    for (int q = 0; q < nq; ++q) { px[m] = quad[2 * q]; py[m] = quad[2 * q + 1]; ++m; }
    if (j < NB) { px[m] = ext_xy[2 * j]; py[m] = ext_xy[2 * j + 1]; ++m; }
    int hx[16], hy[16];
    const int k = small_hull(px, py, m, hx, hy);
    s_k[j] = k;
    for (int q = 0; q < k && q < 8; ++q) { s_px[j][q] = hx[q]; s_py[j][q] = hy[q]; }
    s_c[j] = 0;
  }
  __syncthreads();
  const int2* p2 = reinterpret_cast<const int2*>(xy);
  for (u32 i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int2 p = p2[i];
    for (int j = 0; j <= NB; ++j) {
      const int k = s_k[j];
      bool in = k >= 3;
      for (int q = 0; q < k && in; ++q) {
        const int q2 = q + 1 == k ? 0 : q + 1;
        in = orient64(s_px[j][q], s_py[j][q], s_px[j][q2], s_py[j][q2], p.x, p.y) > 0;
      }
      const u32 bal = __ballot_sync(__activemask(), in);
      if ((threadIdx.x & 31) == (__ffs(__activemask()) - 1) && bal) atomicAdd(&s_c[j], __popc(bal));
    }
  }
  __syncthreads();
  if (threadIdx.x <= NB && s_c[threadIdx.x]) atomicAdd(&counts[threadIdx.x], (unsigned long long)s_c[threadIdx.x]);
}

// ---------------------------------------------------------------- training
// C[M x N] (row-major, ldc = N) = op(A) * op(B) (+ bias[N]) (ReLU) with
// op(A): A (M x K, lda) or A^T; op(B): B^T (B stored N x K) or B (K x N).
// Weights used by the forward pass are rounded to FP16 (round_b).
template <bool TA, bool TB>
__global__ void __launch_bounds__(256)
k_gemm(const float* __restrict__ A, int lda, const float* __restrict__ Bm, int ldb, float* __restrict__ C,
       int M, int N, int K, const float* __restrict__ bias, int relu, int round_b, float beta) {
  __shared__ float sa[16][17], sb[16][17];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int row = blockIdx.y * 16 + ty, col = blockIdx.x * 16 + tx;
  float acc = 0.f;
  for (int k0 = 0; k0 < K; k0 += 16) {
    const int ka = k0 + tx, kb = k0 + ty;
    float av = 0.f, bv = 0.f;
    if (row < M && ka < K) av = TA ? A[(size_t)ka * lda + row] : A[(size_t)row * lda + ka];
    const int bc = blockIdx.x * 16 + tx;
    if (bc < N && kb < K) bv = TB ? Bm[(size_t)kb * ldb + bc] : Bm[(size_t)bc * ldb + kb];
    if (round_b) bv = fp16r(bv);
    sa[ty][tx] = av;
    sb[ty][tx] = bv;
    __syncthreads();
    #pragma unroll
    for (int q = 0; q < 16; ++q) acc = fmaf(sa[ty][q], sb[q][tx], acc);
    __syncthreads();
  }
  if (row < M && col < N) {
    if (bias) acc += round_b ? fp16r(bias[col]) : bias[col];
    if (relu) acc = fmaxf(acc, 0.f);
    C[(size_t)row * N + col] = beta != 0.f ? acc + beta * C[(size_t)row * N + col] : acc;
  }
}

// dZ = 2 (Z - Y) / (B * 32); loss partial sums.
__global__ void k_mse(const float* __restrict__ Z, const float* __restrict__ Y, float* __restrict__ dZ,
                      int count, float scale, float* __restrict__ loss) {
  float l = 0.f;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
    const float d = Z[i] - Y[i];
    dZ[i] = 2.f * d * scale;
    l += d * d;
  }
  #pragma unroll
  for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xFFFFFFFFu, l, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(loss, l * scale);
}

// dH *= (H > 0)
__global__ void k_relu_mask(float* __restrict__ dH, const float* __restrict__ H, int count) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x)
    if (!(H[i] > 0.f)) dH[i] = 0.f;
}

// db[j] = sum over rows of dZ[:, j]
__global__ void k_colsum(const float* __restrict__ dZ, int M, int N, float* __restrict__ db) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= N) return;
  float s = 0.f;
  for (int r = 0; r < M; ++r) s += dZ[(size_t)r * N + j];
  db[j] = s;
}

__global__ void k_adam(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, int count, float lr, float b1, float b2, float eps,
                       float c1, float c2, __half* __restrict__ w16) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi; v[i] = vi;
    const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    w[i] = wi;
    w16[i] = __float2half_rn(wi);
  }
}

__global__ void k_to_half(const float* __restrict__ w, __half* __restrict__ w16, int count) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x)
    w16[i] = __float2half_rn(w[i]);
}

template <bool TA, bool TB>
void gemm(const float* A, int lda, const float* Bm, int ldb, float* C, int M, int N, int K,
          const float* bias, int relu, int round_b, float beta, cudaStream_t st) {
  dim3 grid((N + 15) / 16, (M + 15) / 16);
  k_gemm<TA, TB><<<grid, 256, 0, st>>>(A, lda, Bm, ldb, C, M, N, K, bias, relu, round_b, beta);
}

}  // namespace

int mlp_num_params() { return N_PARAMS; }

cudaError_t launch_features(const int* xy, u32 n, float* feat, int* ext, int* ext_xy, cudaStream_t st) {
  k6_features<<<1, F_BLOCK, 0, st>>>(xy, n, feat, ext, ext_xy);
  return cudaGetLastError();
}

cudaError_t launch_propose(const int* xy, u32 n, const void* w16, float* feat, int* ext, int* ext_xy, Plan* plan,
                           cudaStream_t st) {
  k6_propose<<<1, F_BLOCK, 0, st>>>(xy, n, reinterpret_cast<const __half*>(w16), feat, ext, ext_xy, plan);
  return cudaGetLastError();
}

cudaError_t launch_infer(const float* feat, const void* w16, const int* ext_xy, Plan* plan,
                         cudaStream_t st) {
  k8_infer<<<1, 128, 0, st>>>(feat, reinterpret_cast<const __half*>(w16), ext_xy, plan);
  return cudaGetLastError();
}

cudaError_t launch_labels(const int* xy, u32 n, const int* quad, int nq, const int* ext_xy,
                          unsigned long long* counts, int grid, cudaStream_t st) {
  k10_labels<<<grid, 256, 0, st>>>(xy, n, quad, nq, ext_xy, counts);
  return cudaGetLastError();
}

cudaError_t launch_to_half(const float* w, void* w16, int count, cudaStream_t st) {
  k_to_half<<<64, 256, 0, st>>>(w, reinterpret_cast<__half*>(w16), count);
  return cudaGetLastError();
}

// Forward pass for B feature rows; activations in act = [H1 (B x 128) |
// H2 (B x 128) | Z (B x 32)].
cudaError_t mlp_forward(const float* W, const float* X, int B, float* act, cudaStream_t st) {
  float* H1 = act;
  float* H2 = H1 + (size_t)B * D1;
  float* Z = H2 + (size_t)B * D2;
  gemm<false, false>(X, D0, W + OFF_W1, D0, H1, B, D1, D0, W + OFF_B1, 1, 1, 0.f, st);
  gemm<false, false>(H1, D1, W + OFF_W2, D1, H2, B, D2, D1, W + OFF_B2, 1, 1, 0.f, st);
  gemm<false, false>(H2, D2, W + OFF_W3, D2, Z, B, D3, D2, W + OFF_B3, 0, 1, 0.f, st);
  return cudaGetLastError();
}

// Gradient of the mean squared error (over B x 32 entries) with respect to
// the parameters (evaluated at the FP16-rounded weights); grad and loss are
// overwritten.  scratch holds 2 * B * 128 + B * 32 floats.
cudaError_t mlp_backward(const float* W, const float* X, const float* Y, int B, const float* act,
                         float* grad, float* loss, float* scratch, cudaStream_t st) {
  const float* H1 = act;
  const float* H2 = H1 + (size_t)B * D1;
  const float* Z = H2 + (size_t)B * D2;
  float* dZ = scratch;
  float* dH2 = dZ + (size_t)B * D3;
  float* dH1 = dH2 + (size_t)B * D2;
  cudaMemsetAsync(loss, 0, sizeof(float), st);
  k_mse<<<64, 256, 0, st>>>(Z, Y, dZ, B * D3, 1.f / (float)(B * D3), loss);
  // layer 3
  gemm<true, true>(dZ, D3, H2, D2, grad + OFF_W3, D3, D2, B, nullptr, 0, 0, 0.f, st);
  k_colsum<<<1, D3, 0, st>>>(dZ, B, D3, grad + OFF_B3);
  gemm<false, true>(dZ, D3, W + OFF_W3, D2, dH2, B, D2, D3, nullptr, 0, 1, 0.f, st);
  k_relu_mask<<<64, 256, 0, st>>>(dH2, H2, B * D2);
  // layer 2
  gemm<true, true>(dH2, D2, H1, D1, grad + OFF_W2, D2, D1, B, nullptr, 0, 0, 0.f, st);
  k_colsum<<<1, D2, 0, st>>>(dH2, B, D2, grad + OFF_B2);
  gemm<false, true>(dH2, D2, W + OFF_W2, D1, dH1, B, D1, D2, nullptr, 0, 1, 0.f, st);
  k_relu_mask<<<64, 256, 0, st>>>(dH1, H1, B * D1);
  // layer 1
  gemm<true, true>(dH1, D1, X, D0, grad + OFF_W1, D1, D0, B, nullptr, 0, 0, 0.f, st);
  k_colsum<<<1, D1, 0, st>>>(dH1, B, D1, grad + OFF_B1);
  return cudaGetLastError();
}

cudaError_t mlp_adam(float* W, const float* grad, float* m, float* v, int step, float lr,
                     void* w16, cudaStream_t st) {
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
  k_adam<<<64, 256, 0, st>>>(W, grad, m, v, N_PARAMS, lr, b1, b2, eps, c1, c2,
                             reinterpret_cast<__half*>(w16));
  return cudaGetLastError();
}

}  // namespace gbh
