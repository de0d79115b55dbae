// Device helpers for monotone chains over lexicographically sorted points
// (Section 2.1 step 8), shared by the single-hull finalisation (K5) and the
// batched kernel: accessors, the turn test, the tangent search and the
// warp-cooperative bridge search that merges two adjacent chains.
//
// Two chains over points that are lexicographically separated (every
// point of A before every point of B) merge at their common tangent: with
// t(i) the first j where a_i -> b_j -> b_j+1 turns strictly (the farthest
// tangent point of B seen from a_i), the merged chain keeps a_0..a_i* and
// b_t(i*).. where i* is the first i at which a_i+1 is on or beyond the line
// a_i -> b_t(i).  Both predicates are monotone along convex chains, so a
// warp finds i* by a 32-ary search whose probes each binary-search t.
// sign = +1 builds the lower chain (left turns), -1 the upper chain.
#pragma once

#include "hull_internal.cuh"

namespace gbh {
namespace chain {

struct SmemChain {
  const int* x;
  const int* y;
  __device__ __forceinline__ int2 operator()(int i) const { return make_int2(x[i], y[i]); }
};
struct GlobalChain {
  const int2* xy;
  __device__ __forceinline__ int2 operator()(int i) const { return __ldcg(&xy[i]); }
};

__device__ __forceinline__ long long turn(int sgn, int2 a, int2 b, int2 c) {
  long long o = orient(a.x, a.y, b.x, b.y, c.x, c.y);
  return sgn > 0 ? o : -o;
}

// First j in [0, beta - 1) with a strict turn a -> b_j -> b_j+1, else beta - 1.
template <class Acc>
__device__ __forceinline__ int tangent(const Acc& B, int beta, int2 a, int sgn) {
  int lo = 0, hi = beta - 1;
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (turn(sgn, a, B(mid), B(mid + 1)) > 0) hi = mid;
    else lo = mid + 1;
  }
  return lo;
}

// Warp-cooperative bridge search; all lanes return the same (i*, j*).
template <class AccA, class AccB>
__device__ __forceinline__ void bridge(const AccA& A, int alpha, const AccB& B, int beta, int sgn, int& istar,
                       int& jstar) {
  const int lane = threadIdx.x & 31;
  int lo = 0, hi = alpha - 1;               // the predicate holds at hi
  while (hi > lo) {
    const int span = hi - lo;
    const int q = (span <= 32) ? lo + lane : lo + (int)(((long long)span * lane) >> 5);
    bool pv = true;
    if (q < hi) {
      const int2 a = A(q);
      const int t = tangent(B, beta, a, sgn);
      pv = turn(sgn, a, B(t), A(q + 1)) >= 0;
    }
    const unsigned m = __ballot_sync(0xFFFFFFFFu, pv);
    const int f = m ? (__ffs(m) - 1) : 32;
    const int qprev = __shfl_sync(0xFFFFFFFFu, q, f > 0 ? f - 1 : 0);
    const int qf = __shfl_sync(0xFFFFFFFFu, q, f < 32 ? f : 31);
    if (f == 0) {
      hi = lo;
    } else {
      lo = qprev + 1;
      if (f < 32) hi = qf;
    }
  }
  istar = lo;
  jstar = tangent(B, beta, A(lo), sgn);
}

// The same bridge found by one thread: starting from the last point of A
// and the first of B, step back along A while a_i-1 -> a_i -> b_j does not
// turn strictly and forward along B while a_i -> b_j -> b_j+1 does not,
// until neither moves.  Both junction turns are then strict, so the line
// a_i b_j is a common tangent of the two convex chains and the merged chain
// is the same as bridge()'s.  The walk is short when the bridge lies near
// the junction, as it does for chains of few points.
template <class AccA, class AccB>
__device__ __forceinline__ void walk_bridge(const AccA& A, int alpha, const AccB& B, int beta, int sgn,
                                            int& istar, int& jstar) {
  int i = alpha - 1, j = 0;
  bool moved = true;
  while (moved) {
    moved = false;
    while (i > 0 && turn(sgn, A(i - 1), A(i), B(j)) <= 0) { --i; moved = true; }
    while (j < beta - 1 && turn(sgn, A(i), B(j), B(j + 1)) <= 0) { ++j; moved = true; }
  }
  istar = i;
  jstar = j;
}

// Stack-based chain of l <= K points held in shared memory at [b, b + l),
// built in place (the stack never overtakes the read position).  Returns
// the chain length.
__device__ __forceinline__ int leaf_chain(int* sx, int* sy, int* si, int b, int l, int sgn) {
  int k = 0;
  for (int i = 0; i < l; ++i) {
    const int2 p = make_int2(sx[b + i], sy[b + i]);
    const int pid = si[b + i];
    while (k >= 2 && turn(sgn, make_int2(sx[b + k - 2], sy[b + k - 2]),
                          make_int2(sx[b + k - 1], sy[b + k - 1]), p) <= 0)
      --k;
    sx[b + k] = p.x; sy[b + k] = p.y; si[b + k] = pid;
    ++k;
  }
  return k;
}

#ifndef CHAIN_WALK_MAX
#define CHAIN_WALK_MAX 64
#endif

// Merges nleaf <= blockDim.x leaf chains held in shared memory (leaf l at
// [l * LEAF, ...), cnt[l] points) level by level into one chain at
// [0, cnt[0]).  Every level first finds the bridge of every pair: while the
// chains of a level come from at most CHAIN_WALK_MAX points each, one
// thread per pair with walk_bridge, then one warp per pair (bridge); the
// pair's move (destination, source, count) goes to pairs[] (nleaf / 2 + 1
// entries).  Then the whole block moves the kept part of every right-hand
// chain behind the kept part of its left-hand one, each thread taking one
// slot per round.  Called by every thread of the block.
template <int LEAF>
__device__ __forceinline__ void merge_tree(int* sx, int* sy, int* si, int* cnt, int4* pairs, int nleaf, int sgn) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nthreads = blockDim.x, nwarps = nthreads >> 5;
  for (int step = 1; step < nleaf; step <<= 1) {
    const int npair = (nleaf + 2 * step - 1) / (2 * step);
    if (step * LEAF <= CHAIN_WALK_MAX) {
      for (int p = threadIdx.x; p < npair; p += nthreads) {
        const int la = 2 * p * step, lb = la + step;
        int4 mv = make_int4(0, 0, 0, 0);
        if (lb < nleaf) {
          const int aB = la * LEAF, bB = lb * LEAF;
          const int alpha = cnt[la], beta = cnt[lb];
          SmemChain A{sx + aB, sy + aB}, B{sx + bB, sy + bB};
          int is, js;
          walk_bridge(A, alpha, B, beta, sgn, is, js);
          mv = make_int4(aB + is + 1, bB + js, beta - js, 0);
          cnt[la] = is + 1 + (beta - js);
        }
        pairs[p] = mv;
      }
    } else {
      for (int p = wid; p < npair; p += nwarps) {
        const int la = 2 * p * step, lb = la + step;
        int4 mv = make_int4(0, 0, 0, 0);
        if (lb < nleaf) {
          const int aB = la * LEAF, bB = lb * LEAF;
          const int alpha = cnt[la], beta = cnt[lb];
          SmemChain A{sx + aB, sy + aB}, B{sx + bB, sy + bB};
          int is, js;
          bridge(A, alpha, B, beta, sgn, is, js);
          mv = make_int4(aB + is + 1, bB + js, beta - js, 0);
          if (lane == 0) cnt[la] = is + 1 + (beta - js);
        }
        if (lane == 0) pairs[p] = mv;
      }
    }
    __syncthreads();
    // Rounds of blockDim.x slots in increasing order, as many as the leaves'
    // slots need: a destination never lies after its source, so a round
    // writes nothing a later round reads.
    const int span = 2 * step * LEAF;
    const int rounds = (nleaf * LEAF + nthreads - 1) / nthreads;   // <= LEAF: nleaf <= nthreads
    #pragma unroll
    for (int r = 0; r < LEAF; ++r) {
      if (r >= rounds) break;
      const int q = threadIdx.x + r * nthreads;
      int d = -1, vx = 0, vy = 0, vi = 0;
      if (q < nleaf * LEAF && (q % span) >= step * LEAF) {   // a slot of a right-hand chain
        const int4 mv = pairs[q / span];
        const int off = q - mv.y;
        if (off >= 0 && off < mv.z) { vx = sx[q]; vy = sy[q]; vi = si[q]; d = mv.x + off; }
      }
      __syncthreads();
      if (d >= 0) { sx[d] = vx; sy[d] = vy; si[d] = vi; }
    }
    __syncthreads();
  }
}

}  // namespace chain
}  // namespace gbh
