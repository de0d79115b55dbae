// Host-side launchers of the pipeline kernels (one translation unit each).
#pragma once

#include <cuda_runtime.h>

#include "hull_internal.cuh"

namespace gbh {

struct PlanPatch {
  int new_call;        // bump the epoch, clear the error word, set spin_limit
  int zero_hist;
  int zero_counters;
  int set_s, set_npasses, set_ncorner, set_r;
  u32 spin_limit, s, npasses;
  int ncorner;
  u32 r_lo, r_up;
};

cudaError_t launch_plan_patch(Plan* plan, const PlanPatch& p, cudaStream_t st);
cudaError_t launch_hist(const u64* keys, Plan* plan, int grid, cudaStream_t st);
cudaError_t launch_iota(int* out, u32 m, cudaStream_t st);
cudaError_t launch_gather_sorted(const int2* xy, const u32* ia, const u32* ib, const Plan* plan, int2* out_xy,
                                 int* out_idx, u32 cap, cudaStream_t st);
cudaError_t launch_gather_labels(const int* pos, const int* labels, const u32* count,
                                 u32 skip_first, int* out, u32 cap, cudaStream_t st);

// Resident blocks per SM of the persistent kernels (dynamic tile ids).
cudaError_t k2_occupancy(int* count_blocks, int* write_blocks);
cudaError_t k3_occupancy(int* blocks);
cudaError_t k4_occupancy(int* blocks);

int k1_grid(u32 n, int num_sms);
// sample (optional): receives every kSampleStride-th point, ceil(n / kSampleStride) of them.
cudaError_t launch_k1(const int* xy, u32 n, u32 spin_limit, Plan* plan, ExtPartial* partials,
                      int grid, cudaStream_t st, int2* sample = nullptr);

int k2_tile();
cudaError_t k2_configure();
cudaError_t launch_k2(const int* xy, Plan* plan, u64* keys_out, u32* idx_out, u64* status,
                      unsigned char* mask, int grid_count, int grid_write, cudaStream_t st);

// The fused front (k2_fused.cu): the sample's best witness per witness bin
// and region (wkey: 2 kWitnessBins words, zeroed before the launch; the
// sample from K1), the fused filter writing (key, index) pairs in any order
// with the bins' totals (btot, zeroed; count: also count the first-round
// survivors into the plan), and after the bin scan the move into coarse-bin
// order (ccur: kCoarse cursors, zeroed).  The fused filter's last block also
// writes the bin starts, the groups and the split's cursors (fcur).
cudaError_t fused_configure();
cudaError_t fused_occupancy(int* blocks);
// ncount (device), when given: the candidates are sample[0, *ncount) (the
// single-read front's raw survivors; n then bounds their number).
cudaError_t launch_witness(const int2* sample, u32 n, Plan* plan, u64* wkey, int num_sms, cudaStream_t st,
                           const u32* ncount = nullptr);
// With ncount and imap the points are the single-read front's raw survivors:
// *ncount of them at xy (n bounds the count), their input indices in imap.
cudaError_t launch_k2_fused(const int* xy, u32 n, Plan* plan, const u64* wkey, const int2* sample, u64* okey,
                            u32* oidx, u32* btot, u32* bstart, uint2* groups, u32* fcur, bool count, int grid,
                            cudaStream_t st, const u32* ncount = nullptr, const u32* imap = nullptr);
// The single-read front: the sample polygon (k0_poly.cu), then K1 with that
// polygon as its filter, writing the points on or outside it to (rxy, ridx)
// (count in T->raw_count, which must be zero before k0) and the witness
// sample (every kSampleStride-th point) to `sample`.
cudaError_t launch_poly(const int* xy, u32 n, PolyTab* T, int num_sms, cudaStream_t st);
cudaError_t k1_poly_configure();
cudaError_t launch_k1_poly(const int* xy, u32 n, u32 spin_limit, Plan* plan, ExtPartial* partials, const PolyTab* T,
                           u32* raw_count, int2* rxy, u32* ridx, int num_sms, cudaStream_t st);
cudaError_t launch_place(const u64* ak, const u32* ai, u32 n, Plan* plan, const u32* bstart, u32* ccur, u64* ok,
                         u32* oi, int num_sms, cudaStream_t st);
size_t bucket_smem();
size_t bucket_scratch_words(int blocks);
cudaError_t bucket_configure();
cudaError_t bucket_occupancy(int* blocks);
// Coarse bins (ak, av) spread over their bins into (bk, bv) through the
// bins' cursors (fcur, seeded by the bin scan), with every tile's direction
// aggregates per bin (tagg: 2 split_tile()-tile words per bin of the tile's
// coarse bin, at most ceil(s / split_tile()) + kCoarse tiles) and the first
// tile of every coarse bin (ctiles, kCoarse + 1 words).
int split_tile();
cudaError_t launch_split(const u64* ak, const u32* av, u64* bk, u32* bv, Plan* plan, const u32* bstart, u32* fcur,
                         u64* tagg, u32* ctiles, int grid, cudaStream_t st);
cudaError_t split_occupancy(int* blocks);
cudaError_t launch_bucket_sort(const u64* ak, const u32* av, u64* bk, u32* bv, Plan* plan,
                               const uint2* groups, u32* scratch, int grid, cudaStream_t st);
// The pipeline's bucket sort with the second round: every group's
// direction aggregate into its record of `recs` (one per group, cleared by
// the bin scan) and their exclusive prefixes (one block), then the sort of
// every group with the second round run on it (kept points into the t_*
// staging areas; then launch_group_compact).
// Every bin's exclusive second-round prefix (bpre: 2 words per bin; bagg:
// scratch of kBins + kBinPrefixBlocks word pairs) from the split's tile
// aggregates, and the groups' prefixes in their records.
cudaError_t launch_bin_prefix(Plan* plan, const uint2* groups, void* recs, const u64* tagg, const u32* ctiles,
                              u64* bagg, u64* bpre, cudaStream_t st);
cudaError_t launch_bucket_decide(const u64* ak, const u32* av, u64* bk, u32* bv, Plan* plan, const uint2* groups,
                                 u32* scratch, void* recs, const u64* bpre, int2* t_lo_xy, int* t_lo_idx,
                                 int2* t_up_xy, int* t_up_idx, int2* lo_xy, int* lo_idx, int2* up_xy, int* up_idx,
                                 int grid, cudaStream_t st);
cudaError_t launch_group_compact(Plan* plan, const void* status, const int2* t_lo_xy, const int* t_lo_idx,
                                 const int2* t_up_xy, const int* t_up_idx, int2* lo_xy, int* lo_idx,
                                 int2* up_xy, int* up_idx, int grid, cudaStream_t st);
int array_hist_grid(u32 m, int num_sms);
#ifdef GBH_DEBUG_CHECKS
// Debug builds: checks that both region lists are in strictly increasing (x, y) order.
cudaError_t launch_check_regions(const Plan* plan, const int2* lo_xy, const int2* up_xy, cudaStream_t st);
#endif
cudaError_t launch_array_bins(const u64* keys, const u32* vals, u32 m, Plan* plan,
                              unsigned long long* key_or, u32* rows, u32* bstart, uint2* groups,
                              u64* ok, u32* ov, int grid, cudaStream_t st);

int k3_tile();
size_t k3_dyn_smem();
cudaError_t k3_configure();
cudaError_t launch_k3(const u64* kin, const u32* iin, u64* kout, u32* iout, Plan* plan,
                      u64* status, u32 pass, int grid, cudaStream_t st);

int k4_tile();
size_t k4_status_bytes();
cudaError_t launch_k4(const u64* ka, const u32* ia, const u64* kb, const u32* ib, Plan* plan,
                      void* status, size_t nrec, int2* lo_xy, int* lo_idx, int2* up_xy, int* up_idx,
                      int2* t_lo_xy, int* t_lo_idx, int2* t_up_xy, int* t_up_idx, int grid,
                      cudaStream_t st);

// Section 3.4's chunked second round over a sorted list (one block per
// region; pos_* scratch of m ints each; kept labels into out_*).
cudaError_t launch_k4_chunked(const int2* xy, const int* idx, u32 m, u32 bs, Plan* plan, int* pos_lo, int* pos_up,
                              int* out_lo, int* out_up, cudaStream_t st);
// The mirrored second round over both region lists (one block each), the
// kept points staged in st_* and copied back; r_lo / r_up updated.
cudaError_t launch_k4_reverse(Plan* plan, int2* lo_xy, int* lo_idx, int2* up_xy, int* up_idx, int2* st_lo_xy,
                              int* st_lo_idx, int2* st_up_xy, int* st_up_idx, cudaStream_t st);

int k5_chunk();       // points per chain chunk, at most
int k5_min_chunk();   // and at least (the chunk-count arrays are sized for it)
size_t k5_dyn_smem();
cudaError_t k5_configure(int* max_blocks_per_sm);
cudaError_t launch_k5(const int2* lo_xy, const int* lo_idx, const int2* up_xy, const int* up_idx,
                      Plan* plan, int2* h0_xy, int* h0_idx, int2* h1_xy, int* h1_idx, u32* cnt0,
                      u32* cnt1, int4* jobs, int* out, long long cap, int grid, cudaStream_t st);

struct BatchLaunch {
  const int* xy;
  const long long* offsets;
  const int* order;
  int nb;
  u32* queue;
  const long long* slot0;
  u64* ka; u64* kb; u32* ia; u32* ib;
  int2* lxy; int* lidx; int2* uxy; int* uidx;
  int* out_tmp;
  u32* hcount;
  u32* error;
  const void* w16;   // learned proposal weights, or null
  // The segmented path of the largest instances (mode 0: the whole
  // pipeline per block).  k_seg_ext streams all their tiles first; mode 1
  // reduces every instance's tile extremes into its plan, filter polygon
  // and witness table (rec); k_seg_filter streams the tiles again with
  // the witness test and the polygon; mode 2 gathers every instance's
  // survivors and runs the sort, the second round and the chains.
  int mode;
  const int* tfirst;  // [nb + 1]: first tile of every instance of `order`
  void* text;         // per-tile extremes
  u32* tcnt;          // per-tile survivor counts
  void* rec;          // per-instance plan, polygon edges and witness table
};

int batch_pad();
int seg_tile();             // points per tile of the segmented path
size_t seg_rec_bytes();     // bytes of one instance's record
size_t seg_text_bytes();    // bytes of one tile's extremes
cudaError_t seg_configure(int* occ_ext, int* occ_filter);
cudaError_t launch_seg_ext(const BatchLaunch& L, int ntiles, int grid, cudaStream_t st);
cudaError_t launch_seg_filter(const BatchLaunch& L, int ntiles, int grid, cudaStream_t st);
int batch_max_instance();
size_t batch_smem(int block);
cudaError_t batch_configure(int* occ256, int* occ512);
cudaError_t launch_batch(int block, int grid, const BatchLaunch& L, cudaStream_t st);
cudaError_t launch_batch_output(const u32* hcount, const long long* slot0, const int* out_tmp,
                                int B, long long* out_off, int* out, long long cap, u32* error,
                                int grid, cudaStream_t st);

int mlp_num_params();
cudaError_t launch_features(const int* xy, u32 n, float* feat, int* ext, int* ext_xy, cudaStream_t st);
cudaError_t launch_infer(const float* feat, const void* w16, const int* ext_xy, Plan* plan,
                         cudaStream_t st);
// The pipeline's proposal: the gate on a strided sample (the quadrilateral
// kept when it already discards nearly all of it), else features, inference
// and the learned polygon, in one launch.
cudaError_t launch_propose(const int* xy, u32 n, const void* w16, float* feat, int* ext, int* ext_xy, Plan* plan,
                           cudaStream_t st);
cudaError_t launch_labels(const int* xy, u32 n, const int* quad, int nq, const int* ext_xy,
                          unsigned long long* counts, int grid, cudaStream_t st);
cudaError_t launch_to_half(const float* w, void* w16, int count, cudaStream_t st);
cudaError_t mlp_forward(const float* W, const float* X, int B, float* act, cudaStream_t st);
cudaError_t mlp_backward(const float* W, const float* X, const float* Y, int B, const float* act,
                         float* grad, float* loss, float* scratch, cudaStream_t st);
cudaError_t mlp_adam(float* W, const float* grad, float* m, float* v, int step, float lr,
                     void* w16, cudaStream_t st);

// The paper's angular ordering (angular.cu): pass-1 pairs (squared distance
// to the anchor, index) of the first-round survivors keep[0 .. s) and the
// count of points equal to the anchor (n_same, incremented); pass-2 pairs
// (angle key, pass-1 rank) in pass-1 order; the order ([anchor, points by
// angle], m1 entries) as indices and coordinates; P_longest (lpos) and the
// two walks of Figure 2 into keep flags (m1 >= 2; scratch of
// angle_walk_scratch_bytes(m1) bytes).
cudaError_t launch_angle_dist(const int2* xy, const int* keep, u32 s, u32 anchor, u64* keys, u32* vals, u32* n_same,
                              int num_sms, cudaStream_t st);
cudaError_t launch_angle_keys(const int2* xy, const u64* dkeys, const u32* dvals, u32 s, u32 anchor, u64* keys,
                              u32* vals, int num_sms, cudaStream_t st);
cudaError_t launch_angle_order(const int2* xy, const u32* dvals, const u32* avals, u32 m1, u32 anchor, int* order,
                               int2* pts, int num_sms, cudaStream_t st);
size_t angle_walk_scratch_bytes(u32 m1);
// Step 8 of the angular variant: the kept positions of keep[0 .. m1) into
// pos (unordered, count in cnt); phase 0 turns them into (position,
// position) pairs for the sort, phase 1 gathers the points and input
// indices of the sorted positions (vals); the hull's positions out_c[0 .. h)
// mapped to input indices.
cudaError_t launch_angle_compact(const unsigned char* keep, u32 m1, u32* pos, u32* cnt, int num_sms, cudaStream_t st);
cudaError_t launch_angle_gather(const int2* xy, const int* order, u32* pos, u32 r, u64* keys, u32* vals, int2* xy_c,
                                int* lab, int num_sms, cudaStream_t st, int phase);
cudaError_t launch_angle_label(const int* out_c, const int* lab, u32 h, int* out, int num_sms, cudaStream_t st);
cudaError_t launch_angle_walks(const int2* pts, u32 m1, void* scratch, u32* lpos, unsigned char* keep, int num_sms,
                               cudaStream_t st);

}  // namespace gbh
