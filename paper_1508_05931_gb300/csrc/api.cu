// The C ABI (include/gbhull.h): contexts, workspace, argument checks, the
// launch sequence of the pipeline and the per-stage entry points.
#include <algorithm>
#include <cstddef>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <sys/stat.h>
#include <numeric>
#include <string>
#include <vector>

#include "../../include/gbhull.h"
#include "hull_internal.cuh"
#include "kernels.h"

using namespace gbh;

namespace {

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Device workspace for up to `cap` points, carved out of one allocation.
struct Workspace {
  size_t cap = 0;
  void* base = nullptr;
  ExtPartial* partials = nullptr;
  u64* keys[2] = {nullptr, nullptr};
  u32* idx[2] = {nullptr, nullptr};
  u64* st_filter = nullptr;
  u64* st_sort = nullptr;
  void* st_region = nullptr;
  int2* lo_xy = nullptr; int* lo_idx = nullptr;
  int2* up_xy = nullptr; int* up_idx = nullptr;
  int2* h_xy[2] = {nullptr, nullptr};
  int* h_idx[2] = {nullptr, nullptr};
  u32* cnt[2] = {nullptr, nullptr};
  int4* jobs = nullptr;
  int* aux = nullptr;          // int32[cap]: labels for stage entry points
  unsigned char* mask = nullptr;  // first-round keep bits, one byte per 8 points
  // bucket sort
  u32* rows = nullptr;         // per-block bin counts, then prefixes: [rows_cap][kBins]
  size_t rows_cap = 0;
  u32* bstart = nullptr;       // first position of every bin
  uint2* groups = nullptr;     // (first position, first bin) per group, closing record
  u32* bscratch = nullptr;     // per-block scratch of the large-bin split
  u64* tagg = nullptr;         // per split tile and bin: direction aggregates (lower, upper)
  u32* ctiles = nullptr;       // first split tile of every coarse bin
  u32* bcnt = nullptr;         // bins' totals, then coarse-bin cursors (k2_count)
  u64* bagg = nullptr;         // per bin: prefix within its k_bin_prefix block (lower, upper), then block totals
  u64* bpre = nullptr;         // per bin: exclusive second-round prefix (lower, upper)
  u32* fcur = nullptr;         // per bin: next position of the coarse-to-fine split
  u64* wkey = nullptr;         // per region and witness bin: the sample's best witness (follows bcnt)
  int2* sample = nullptr;      // every kSampleStride-th point (K1 or k0 copies them out)
  PolyTab* poly = nullptr;     // the single-read front's sample polygon (follows wkey)
  unsigned long long* key_or = nullptr;
};

struct HostStage {
  size_t cap = 0;
  int32_t* d_in = nullptr;     // device copy of host points
  int32_t* d_out = nullptr;    // device output for host calls
  int32_t* d_in2 = nullptr;    // second input buffer of hull_compute_host_multi (same cap)
  cudaStream_t copy = nullptr; // copy stream of hull_compute_host_multi
  cudaEvent_t copied[2] = {nullptr, nullptr}, consumed[2] = {nullptr, nullptr};
};

// Workspace of the batched kernels: per-instance scratch slots and tables.
struct BatchWs {
  size_t cap_slots = 0, cap_b = 0;
  void* base = nullptr;
  u64* ka = nullptr; u64* kb = nullptr; u32* ia = nullptr; u32* ib = nullptr;
  int2* lxy = nullptr; int* lidx = nullptr; int2* uxy = nullptr; int* uidx = nullptr;
  int* out_tmp = nullptr;
  long long* slot0 = nullptr;
  int* order = nullptr;
  u32* hcount = nullptr;
  u32* ctl = nullptr;          // [0], [1]: queues; [2]: error bits
  // pinned host staging
  size_t h_cap = 0;
  long long* h_off = nullptr;
  long long* h_slot0 = nullptr;
  int* h_order = nullptr;
  int* h_tfirst = nullptr;
  u32* h_ctl = nullptr;
  // segmented path of the largest instances: tile extremes and counts,
  // per-instance records, first tile of every instance
  size_t cap_tiles = 0, cap_seg = 0;
  void* seg = nullptr;
  void* text = nullptr;
  u32* tcnt = nullptr;
  void* rec = nullptr;
  int* tfirst = nullptr;
};

constexpr int64_t kSmallInstance = 16384;   // size bucket boundary
// Instances of this many points or more take the segmented path (flat
// streaming passes over all their tiles) unless the autotuner chose another
// boundary among kSegCandidates (the last one: no instance takes it).
constexpr int64_t kSegDefault = 65536;
constexpr int64_t kSegOff = (int64_t)1 << 40;
constexpr int64_t kSegCandidates[4] = {32768, 131072, 262144, kSegOff};

}  // namespace

struct hull_ctx {
  int device = 0;
  hull_config cfg{};
  int num_sms = 0;
  int occ_k2c = 1, occ_k2 = 1, occ_k3 = 1, occ_k4 = 1, occ_k5 = 1;
  int occ_kb = 1, occ_sp = 1;  // bucket sort: group sort, split
  int occ_kf = 1;              // the fused filter
  Plan* plan = nullptr;        // device
  Plan* h_plan = nullptr;      // pinned host mirror of the summary fields
  char* h_multi = nullptr;     // pinned summaries of hull_compute_multi (one per input)
  int32_t h_multi_cap = 0;
  Workspace ws;
  // Second lane of hull_compute_multi: its own workspace and Plan, used on
  // the aux stream while lane 0 runs on the caller's stream.
  Workspace ws2;
  Plan* plan2 = nullptr;
  // Scratch of the angular variant (hull_stage_angular and
  // hull_compute_angular): grown to the largest call, kept.
  void* ang = nullptr;
  size_t ang_bytes = 0;
  HostStage hs;
  hull_stats last{};
  int64_t fallbacks = 0;       // calls rerun on the radix passes
  // stage timing (hull_set_profiling)
  bool prof = false;
  bool prof_pending = false;
  cudaEvent_t ev[HULL_NUM_STAGES + 1] = {};
  hull_profile profile{};
  // batched mode
  BatchWs bw;
  cudaStream_t aux = nullptr;
  cudaEvent_t bev[2] = {nullptr, nullptr};
  int occ_b256 = 1, occ_b512 = 1;
  int occ_sx = 1, occ_sf = 1;   // segmented streaming passes
  int tuned_block[3] = {0, 0, 0};  // per bucket (small, large, segmented); 0 = not tuned yet
  int64_t tuned_seg = 0;        // smallest instance of the segmented path; 0 = not tuned yet
  // learned proposal
  bool have_weights = false;
  float* W = nullptr;           // FP32 master parameters
  void* W16 = nullptr;          // FP16 copies used by inference / forward
  float* adam_m = nullptr;
  float* adam_v = nullptr;
  int adam_step = 0;
  float* feat = nullptr;        // 64 features
  int* ext = nullptr;           // 32 direction extremes (indices)
  int* ext_xy = nullptr;        // and their coordinates
  unsigned long long* lab_cnt = nullptr;   // 33 label counters
  float* d_loss = nullptr;
  float* grad = nullptr;
  size_t train_cap = 0;         // rows of the training scratch
  float* act = nullptr;
  float* scratch = nullptr;
};

namespace {

constexpr size_t kSummaryBytes = offsetof(Plan, ctr);

hull_status cuda_fail(cudaError_t e) {
  (void)e;
  cudaGetLastError();   // clear a non-sticky error so the context stays usable
  return HULL_ECUDA;
}

struct DevGuard {
  int prev = -1;
  explicit DevGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DevGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

void free_ws(Workspace& w) {
  if (w.base) cudaFree(w.base);
  w = Workspace{};
}

hull_status ensure_ws(hull_ctx* c, size_t n) {
  if (n <= c->ws.cap && c->ws.base) return HULL_OK;
  size_t cap = align_up(n < 65536 ? 65536 : n, 65536);
  const size_t chunk = (size_t)k5_chunk();
  const size_t t2 = (cap + k2_tile() - 1) / k2_tile() + 1;
  const size_t t3 = (cap + k3_tile() - 1) / k3_tile() + 1;
  const size_t t4 = (cap + k4_tile() - 1) / k4_tile() + 1;
  const size_t slots = cap + 4 + 2 * chunk;
  const size_t nchunks = slots / (size_t)k5_min_chunk() + 2;
  const size_t parts = (size_t)c->num_sms * 4 + 8;
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t o = off; off = align_up(off + bytes, 256); return o; };
  const size_t o_part = take(parts * sizeof(ExtPartial));
  // Key and index arrays have 64 bytes to spare past their end: the bucket
  // sort's bulk copies round their sizes up to 16 bytes.
  const size_t o_k0 = take(cap * 8 + 64), o_k1 = take(cap * 8 + 64);
  const size_t o_i0 = take(cap * 4 + 64), o_i1 = take(cap * 4 + 64);
  const size_t o_sf = take(t2 * 8), o_ss = take(t3 * kRadix * 8);
  // Look-back records of K4's chunks, or of the bucket sort's groups (at most one per bin).
  const size_t o_sr = take(std::max(t4, (size_t)kBins + 2) * k4_status_bytes());
  const size_t status_end = off;
  const size_t o_lxy = take((cap + 2) * 8), o_lid = take((cap + 2) * 4);
  const size_t o_uxy = take((cap + 2) * 8), o_uid = take((cap + 2) * 4);
  const size_t o_h0x = take(slots * 8), o_h0i = take(slots * 4);
  const size_t o_h1x = take(slots * 8), o_h1i = take(slots * 4);
  const size_t o_c0 = take(nchunks * 4), o_c1 = take(nchunks * 4);
  const size_t o_jobs = take(nchunks * 16);
  const size_t o_aux = take(cap * 4);
  const size_t o_mask = take(cap / 8 + 4096);
  const size_t rows_cap = (size_t)c->num_sms * 2;   // histogram rows of the array sort (array_hist_grid)
  const size_t o_rows = take(rows_cap * kBins * 4);
  const size_t o_bstart = take((size_t)kBins * 4);
  const size_t o_groups = take(((size_t)kBins + 2) * 8);
  const size_t o_bscr = take(bucket_scratch_words(c->num_sms * c->occ_kb) * 4);
  const size_t o_kor = take(8);
  const size_t tiles_cap = cap / (size_t)split_tile() + (size_t)kCoarse + 1;
  const size_t o_tagg = take(tiles_cap * 2 * kFinePerCoarse * 8);
  const size_t o_ctiles = take(((size_t)kCoarse + 1) * 4);
  const size_t o_bcnt = take(((size_t)kBins + kCoarse) * 4);
  const size_t o_wkey = take((size_t)2 * kWitnessBins * 8);   // right after bcnt: one memset clears both
  const size_t o_poly = take(sizeof(PolyTab));                 // right after wkey: the same memset clears its head
  const size_t o_sample = take((cap / kSampleStride + 1) * 8);
  const size_t o_bagg = take(((size_t)kBins + kBinPrefixBlocks) * 16);
  const size_t o_bpre = take((size_t)kBins * 16);
  const size_t o_fcur = take((size_t)kBins * 4);
  const size_t total = off;

  cudaDeviceSynchronize();
  free_ws(c->ws);
  void* base = nullptr;
  if (cudaMalloc(&base, total) != cudaSuccess) {
    cudaGetLastError();
    return HULL_ENOMEM;
  }
  // Look-back status words must start out matching no epoch.
  if (cudaMemset(base, 0, status_end) != cudaSuccess) {
    cudaFree(base);
    return cuda_fail(cudaErrorUnknown);
  }
  char* b = static_cast<char*>(base);
  Workspace& w = c->ws;
  w.cap = cap;
  w.base = base;
  w.partials = reinterpret_cast<ExtPartial*>(b + o_part);
  w.keys[0] = reinterpret_cast<u64*>(b + o_k0); w.keys[1] = reinterpret_cast<u64*>(b + o_k1);
  w.idx[0] = reinterpret_cast<u32*>(b + o_i0);  w.idx[1] = reinterpret_cast<u32*>(b + o_i1);
  w.st_filter = reinterpret_cast<u64*>(b + o_sf);
  w.st_sort = reinterpret_cast<u64*>(b + o_ss);
  w.st_region = b + o_sr;
  w.lo_xy = reinterpret_cast<int2*>(b + o_lxy); w.lo_idx = reinterpret_cast<int*>(b + o_lid);
  w.up_xy = reinterpret_cast<int2*>(b + o_uxy); w.up_idx = reinterpret_cast<int*>(b + o_uid);
  w.h_xy[0] = reinterpret_cast<int2*>(b + o_h0x); w.h_idx[0] = reinterpret_cast<int*>(b + o_h0i);
  w.h_xy[1] = reinterpret_cast<int2*>(b + o_h1x); w.h_idx[1] = reinterpret_cast<int*>(b + o_h1i);
  w.cnt[0] = reinterpret_cast<u32*>(b + o_c0); w.cnt[1] = reinterpret_cast<u32*>(b + o_c1);
  w.jobs = reinterpret_cast<int4*>(b + o_jobs);
  w.aux = reinterpret_cast<int*>(b + o_aux);
  w.mask = reinterpret_cast<unsigned char*>(b + o_mask);
  w.rows = reinterpret_cast<u32*>(b + o_rows);
  w.rows_cap = rows_cap;
  w.bstart = reinterpret_cast<u32*>(b + o_bstart);
  w.groups = reinterpret_cast<uint2*>(b + o_groups);
  w.bscratch = reinterpret_cast<u32*>(b + o_bscr);
  w.key_or = reinterpret_cast<unsigned long long*>(b + o_kor);
  w.tagg = reinterpret_cast<u64*>(b + o_tagg);
  w.ctiles = reinterpret_cast<u32*>(b + o_ctiles);
  w.bcnt = reinterpret_cast<u32*>(b + o_bcnt);
  w.bagg = reinterpret_cast<u64*>(b + o_bagg);
  w.bpre = reinterpret_cast<u64*>(b + o_bpre);
  w.fcur = reinterpret_cast<u32*>(b + o_fcur);
  w.wkey = reinterpret_cast<u64*>(b + o_wkey);
  w.poly = reinterpret_cast<PolyTab*>(b + o_poly);
  w.sample = reinterpret_cast<int2*>(b + o_sample);
  return HULL_OK;
}

int grid_for(int occ, int num_sms, size_t work_tiles) {
  size_t g = (size_t)occ * (size_t)num_sms;
  if (work_tiles < g) g = work_tiles;
  if (g < 1) g = 1;
  return (int)g;
}

// Copies the summary back, synchronises and maps device error bits.  With
// `fallback`, a bucket sort that met a bin too large for it (ERR_FALLBACK,
// no other error) sets *fallback and returns HULL_OK without recording
// anything: the caller reruns the call on the radix passes.
hull_status read_summary(hull_ctx* c, const Plan& p, bool* fallback);

hull_status finish(hull_ctx* c, cudaStream_t st, bool* fallback = nullptr) {
  cudaError_t e = cudaMemcpyAsync(c->h_plan, c->plan, kSummaryBytes, cudaMemcpyDeviceToHost, st);
  if (e != cudaSuccess) return cuda_fail(e);
  e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e);
  return read_summary(c, *c->h_plan, fallback);
}

// The bookkeeping of finish() for one call's summary `p` (already on the host).
hull_status read_summary(hull_ctx* c, const Plan& p, bool* fallback) {
  if (fallback) {
    *fallback = (p.error & ERR_FALLBACK) != 0 && (p.error & (ERR_RANGE | ERR_TIMEOUT)) == 0;
    if (*fallback) return HULL_OK;
  }
  if (c->prof_pending) {
    c->prof_pending = false;
    hull_profile& f = c->profile;
    for (int k = 0; k < HULL_NUM_STAGES; ++k) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, c->ev[k], c->ev[k + 1]) == cudaSuccess) f.ms[k] += ms;
    }
    cudaGetLastError();
    f.calls += 1;
    f.radix_calls += p.sorted_in_b && p.ngroups ? 0 : 1;
    f.sort_passes += p.npasses;
    f.points += p.n;
    f.survivors += p.s_quad;
    f.raw_survivors += p.s_raw;
    f.single_read_calls += p.s_raw ? 1 : 0;
    f.second_round += (int64_t)p.r_lo + p.r_up;
    f.witness_survivors += p.s;
  }
  if (c->cfg.collect_stats) {
    c->last.n = p.n; c->last.s = p.s_quad; c->last.s_witness = p.s;
    c->last.r_lower = p.r_lo; c->last.r_upper = p.r_up;
    c->last.h = p.h;
    for (int j = 0; j < 4; ++j) c->last.ext[j] = p.ext_idx[j];
    c->last.ncorner = p.ncorner;
  }
  c->last.learned_used = p.learned_used;
  if (p.error & ERR_RANGE) return HULL_ERANGE;
  if (p.error & ERR_TIMEOUT) return HULL_ETIMEOUT;
  if (p.error & ERR_INTERNAL) return HULL_EINTERNAL;
  if (p.error & ERR_CAPACITY) return HULL_ECAPACITY;
  return HULL_OK;
}

bool aligned8(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 7u) == 0; }

void mark(hull_ctx* c, int k, cudaStream_t st) {
  if (c->prof_pending) cudaEventRecord(c->ev[k], st);
}

// Inputs from this size up (16-byte aligned, no statistics asked for) take
// the single-read front on the bucket-sort path.
constexpr u32 kSingleReadMin = 1u << 16;

// K1 .. K4 of the pipeline on d_xy (n >= 1).  `bucket` selects the bucket
// sort (K2 scatters the survivors into bins, one block sorts each group of
// bins); otherwise K2 compacts them in index order for the radix passes.
// `exact_lists`: the region lists must be exactly Figure 2's on every
// first-round survivor (the two-read front; the single-read front's lists
// are Figure 2's on a subset of them, which keeps every hull vertex).
hull_status run_front(hull_ctx* c, const int32_t* d_xy, u32 n, cudaStream_t st, bool bucket,
                      bool exact_lists = false) {
  Workspace& w = c->ws;
  const bool single = bucket && !exact_lists && !c->cfg.collect_stats && n >= kSingleReadMin &&
                      (reinterpret_cast<uintptr_t>(d_xy) & 15u) == 0;
  const size_t clear_bytes = (reinterpret_cast<char*>(w.wkey) - reinterpret_cast<char*>(w.bcnt)) +
                             (size_t)2 * kWitnessBins * sizeof(u64) + kPolyClearBytes;
  mark(c, 0, st);
  cudaError_t e = cudaSuccess;
  if (single) {
    // The single-read front: the sample polygon (from every 1024th point),
    // then one pass for the extremes that drops the points strictly inside
    // that polygon and writes the rest (raw survivors, ~0.1-1 % of a uniform
    // input) to the chain buffers, free until the group sort; the raw
    // survivors are also the witnesses' candidates.
    e = cudaMemsetAsync(w.bcnt, 0, clear_bytes, st);
    if (e == cudaSuccess) e = launch_poly(d_xy, n, w.poly, c->num_sms, st);
    mark(c, 1, st);
    if (e == cudaSuccess)
      e = launch_k1_poly(d_xy, n, c->cfg.spin_limit, c->plan, w.partials, w.poly, &w.poly->raw_count, w.h_xy[0],
                         reinterpret_cast<u32*>(w.h_idx[0]), c->num_sms, st);
  } else {
    if (bucket) mark(c, 1, st);     // no sample polygon: an empty stage
    e = launch_k1(d_xy, n, c->cfg.spin_limit, c->plan, w.partials, k1_grid(n, c->num_sms), st,
                  bucket ? w.sample : nullptr);
  }
  if (e != cudaSuccess) return cuda_fail(e);
  if (c->cfg.proposal == 1 && c->have_weights && !single) {
    // Learned filter polygon: sampled features, MLP, exact hull of the
    // chosen extremes and the quadrilateral's corners, unless the gate finds
    // the quadrilateral already discarding nearly all of a sample.  Not on
    // the single-read front: there the filter polygon only meets the raw
    // survivors of the sample polygon (32 directions) after the witness
    // test, and a larger polygon cannot pay for its features and inference.
    e = launch_propose(d_xy, n, c->W16, c->feat, c->ext, c->ext_xy, c->plan, st);
    if (e != cudaSuccess) return cuda_fail(e);
  }
  mark(c, bucket ? 2 : 1, st);
  const size_t t2 = (n + k2_tile() - 1) / k2_tile();
  if (bucket) {
    // The fused front: witnesses from a sample, then one pass that filters,
    // tests every first-round survivor against its bin's witness and
    // compacts what is left with the bins' totals; the bin starts and groups;
    // the survivors moved into coarse-bin order.  Then the split into bins
    // (with their direction aggregates), every bin's and group's prefix, and
    // one block per group of bins sorts it in shared memory and runs the
    // second round on it from its prefix.
    // Profile slots: 0 sample polygon, 1 extremes, 2 witnesses, 3 filter
    // (the fused filter and its bin scan), 4 scatter (coarse bins), 5 split
    // (fine bins, their aggregates, group prefixes), 6 sort (+ second
    // round), 7..9 empty, 10 compaction.
    if (!single) e = cudaMemsetAsync(w.bcnt, 0, clear_bytes, st);
    // Witnesses: on the single-read front from every raw survivor (the
    // points nearest the hull, a small fraction of the input), else from
    // the every-32nd-point sample.
    const int2* wsrc = single ? reinterpret_cast<const int2*>(w.h_xy[0]) : w.sample;
    if (e == cudaSuccess)
      e = launch_witness(wsrc, n, c->plan, w.wkey, c->num_sms, st, single ? &w.poly->raw_count : nullptr);
    if (e != cudaSuccess) return cuda_fail(e);
    mark(c, 3, st);
    if (single)   // the fused filter over the raw survivors, indices mapped back to the input's
      e = launch_k2_fused(reinterpret_cast<const int*>(w.h_xy[0]), n, c->plan, w.wkey, wsrc, w.keys[1], w.idx[1],
                          w.bcnt, w.bstart, w.groups, w.fcur, false, c->occ_kf * c->num_sms, st, &w.poly->raw_count,
                          reinterpret_cast<const u32*>(w.h_idx[0]));
    else
      e = launch_k2_fused(d_xy, n, c->plan, w.wkey, w.sample, w.keys[1], w.idx[1], w.bcnt, w.bstart, w.groups,
                          w.fcur, c->cfg.collect_stats != 0, c->occ_kf * c->num_sms, st);
    if (e != cudaSuccess) return cuda_fail(e);
    mark(c, 4, st);
    e = launch_place(w.keys[1], w.idx[1], n, c->plan, w.bstart, w.bcnt + kBins, w.keys[0], w.idx[0], c->num_sms, st);
    if (e != cudaSuccess) return cuda_fail(e);
    mark(c, 5, st);
    e = launch_split(w.keys[0], w.idx[0], w.keys[1], w.idx[1], c->plan, w.bstart, w.fcur, w.tagg, w.ctiles,
                     c->occ_sp * c->num_sms, st);
    if (e == cudaSuccess) e = launch_bin_prefix(c->plan, w.groups, w.st_region, w.tagg, w.ctiles, w.bagg, w.bpre, st);
    if (e != cudaSuccess) return cuda_fail(e);
    mark(c, 6, st);
    e = launch_bucket_decide(w.keys[1], w.idx[1], w.keys[0], w.idx[0], c->plan, w.groups, w.bscratch,
                             w.st_region, w.bpre, w.h_xy[0], w.h_idx[0], w.h_xy[1], w.h_idx[1], w.lo_xy, w.lo_idx,
                             w.up_xy, w.up_idx, c->occ_kb * c->num_sms, st);
    if (e != cudaSuccess) return cuda_fail(e);
    for (int p = 7; p <= 2 + kMaxPasses; ++p) mark(c, p, st);
    e = launch_group_compact(c->plan, w.st_region, w.h_xy[0], w.h_idx[0], w.h_xy[1], w.h_idx[1], w.lo_xy,
                             w.lo_idx, w.up_xy, w.up_idx, grid_for(c->occ_k4, c->num_sms, kBins), st);
    if (e != cudaSuccess) return cuda_fail(e);
#ifdef GBH_DEBUG_CHECKS
    e = launch_check_regions(c->plan, w.lo_xy, w.up_xy, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e);
#endif
    if (c->cfg.reverse_round) {
      e = launch_k4_reverse(c->plan, w.lo_xy, w.lo_idx, w.up_xy, w.up_idx, w.h_xy[0], w.h_idx[0], w.h_xy[1],
                            w.h_idx[1], st);
      if (e != cudaSuccess) return cuda_fail(e);
    }
    mark(c, 3 + kMaxPasses, st);
    return HULL_OK;
  } else {
    e = launch_k2(d_xy, c->plan, w.keys[0], w.idx[0], w.st_filter, w.mask, grid_for(c->occ_k2c, c->num_sms, t2),
                  grid_for(c->occ_k2, c->num_sms, t2), st);
    if (e != cudaSuccess) return cuda_fail(e);
    mark(c, 2, st);
    const size_t t3 = (n + k3_tile() - 1) / k3_tile();
    for (u32 p = 0; p < (u32)kMaxPasses; ++p) {
      e = launch_k3(w.keys[p & 1], w.idx[p & 1], w.keys[(p + 1) & 1], w.idx[(p + 1) & 1], c->plan,
                    w.st_sort, p, grid_for(c->occ_k3, c->num_sms, t3), st);
      if (e != cudaSuccess) return cuda_fail(e);
      mark(c, 3 + (int)p, st);
    }
  }
  const size_t t4 = (n + k4_tile() - 1) / k4_tile();
  e = launch_k4(w.keys[0], w.idx[0], w.keys[1], w.idx[1], c->plan, w.st_region, t4, w.lo_xy, w.lo_idx,
                w.up_xy, w.up_idx, w.h_xy[0], w.h_idx[0], w.h_xy[1], w.h_idx[1],
                grid_for(c->occ_k4, c->num_sms, t4), st);
  if (e == cudaSuccess && c->cfg.reverse_round)
    e = launch_k4_reverse(c->plan, w.lo_xy, w.lo_idx, w.up_xy, w.up_idx, w.h_xy[0], w.h_idx[0], w.h_xy[1], w.h_idx[1],
                          st);
  if (e != cudaSuccess) return cuda_fail(e);
  mark(c, 3 + kMaxPasses, st);
  return HULL_OK;
}

hull_status run_final(hull_ctx* c, const int2* lo_xy, const int* lo_idx, const int2* up_xy,
                      const int* up_idx, size_t npoints_bound, int32_t* d_out, int64_t cap,
                      cudaStream_t st) {
  Workspace& w = c->ws;
  const size_t chunks = (npoints_bound + 4) / (size_t)k5_chunk() + 2;
  int grid = grid_for(c->occ_k5 < 4 ? c->occ_k5 : 4, c->num_sms, chunks < 64 ? 64 : chunks);
  cudaError_t e = launch_k5(lo_xy, lo_idx, up_xy, up_idx, c->plan, w.h_xy[0], w.h_idx[0], w.h_xy[1],
                            w.h_idx[1], w.cnt[0], w.cnt[1], w.jobs, d_out, (long long)cap, grid, st);
  if (e != cudaSuccess) return cuda_fail(e);
  mark(c, 4 + kMaxPasses, st);
  return HULL_OK;
}

hull_status new_call_patch(hull_ctx* c, cudaStream_t st, PlanPatch p) {
  p.new_call = 1;
  p.spin_limit = c->cfg.spin_limit;
  p.zero_counters = 1;
  cudaError_t e = launch_plan_patch(c->plan, p, st);
  return e == cudaSuccess ? HULL_OK : cuda_fail(e);
}

std::string autotune_path() {
  const char* p = std::getenv("GBHULL_AUTOTUNE_CACHE");
  if (p && *p) return p;
  const char* h = std::getenv("HOME");
  return std::string(h && *h ? h : "/tmp") + "/.cache/gbhull_autotune.json";
}

std::string device_key(const hull_ctx* c) {
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, c->device) != cudaSuccess) return "unknown";
  int drv = 0;
  cudaDriverGetVersion(&drv);
  std::string k = prop.name;
  for (char& ch : k)
    if (ch == '"' || ch == '\\') ch = '_';
  return k + "/sm" + std::to_string(prop.major) + std::to_string(prop.minor) + "/drv" + std::to_string(drv);
}

// The cache is a flat JSON object {"<device>|batched_small": 256, ...}.
void autotune_load(hull_ctx* c) {
  FILE* f = std::fopen(autotune_path().c_str(), "r");
  if (!f) return;
  std::string txt;
  char buf[4096];
  size_t r;
  while ((r = std::fread(buf, 1, sizeof(buf), f)) > 0) txt.append(buf, r);
  std::fclose(f);
  const std::string dk = device_key(c);
  const char* names[3] = {"batched_small", "batched_large", "batched_seg_block"};
  for (int b = 0; b < 3; ++b) {
    const std::string key = "\"" + dk + "|" + names[b] + "\":";
    const size_t pos = txt.find(key);
    if (pos == std::string::npos) continue;
    const int v = std::atoi(txt.c_str() + pos + key.size());
    if (v == 256 || v == 512) c->tuned_block[b] = v;
  }
  const std::string key = "\"" + dk + "|batched_seg_min\":";
  const size_t pos = txt.find(key);
  if (pos != std::string::npos) {
    const long long v = std::atoll(txt.c_str() + pos + key.size());
    for (int64_t cand : kSegCandidates)
      if (v == cand) c->tuned_seg = v;
    if (v == kSegDefault) c->tuned_seg = v;
  }
}

void autotune_save(const hull_ctx* c) {
  const std::string path = autotune_path();
  const size_t slash = path.find_last_of('/');
  if (slash != std::string::npos && slash > 0) mkdir(path.substr(0, slash).c_str(), 0755);
  FILE* f = std::fopen(path.c_str(), "w");
  if (!f) return;
  const std::string dk = device_key(c);
  std::fprintf(f, "{\"%s|batched_small\": %d, \"%s|batched_large\": %d, \"%s|batched_seg_block\": %d",
               dk.c_str(), c->tuned_block[0] ? c->tuned_block[0] : 256, dk.c_str(),
               c->tuned_block[1] ? c->tuned_block[1] : 256, dk.c_str(), c->tuned_block[2] ? c->tuned_block[2] : 256);
  if (c->tuned_seg) std::fprintf(f, ", \"%s|batched_seg_min\": %lld", dk.c_str(), (long long)c->tuned_seg);
  std::fprintf(f, "}\n");
  std::fclose(f);
}

// Device staging for the host entry points: input and output buffers of at
// least n points (two input buffers, a copy stream and its events with
// `pipelined`).  Growing synchronises the device.
hull_status ensure_host_stage(hull_ctx* c, size_t n, bool pipelined) {
  HostStage& hs = c->hs;
  if (n > hs.cap || (pipelined && !hs.d_in2)) {
    cudaDeviceSynchronize();
    const size_t hc = align_up(n > hs.cap ? n : hs.cap, 65536);
    if (hs.d_in) cudaFree(hs.d_in);
    if (hs.d_out) cudaFree(hs.d_out);
    if (hs.d_in2) cudaFree(hs.d_in2);
    hs.d_in = hs.d_out = hs.d_in2 = nullptr;
    hs.cap = 0;
    bool ok = cudaMalloc(&hs.d_in, hc * 8) == cudaSuccess && cudaMalloc(&hs.d_out, hc * 4) == cudaSuccess;
    if (ok && pipelined) ok = cudaMalloc(&hs.d_in2, hc * 8) == cudaSuccess;
    if (!ok) {
      cudaGetLastError();
      if (hs.d_in) cudaFree(hs.d_in);
      if (hs.d_out) cudaFree(hs.d_out);
      if (hs.d_in2) cudaFree(hs.d_in2);
      hs.d_in = hs.d_out = hs.d_in2 = nullptr;
      return HULL_ENOMEM;
    }
    hs.cap = hc;
  }
  if (pipelined && !hs.copy) {
    if (cudaStreamCreateWithFlags(&hs.copy, cudaStreamNonBlocking) != cudaSuccess) return cuda_fail(cudaErrorUnknown);
    for (int k = 0; k < 2; ++k)
      if (cudaEventCreateWithFlags(&hs.copied[k], cudaEventDisableTiming) != cudaSuccess ||
          cudaEventCreateWithFlags(&hs.consumed[k], cudaEventDisableTiming) != cudaSuccess)
        return cuda_fail(cudaErrorUnknown);
  }
  return HULL_OK;
}

}  // namespace

extern "C" {

const char* hull_status_string(hull_status s) {
  switch (s) {
    case HULL_OK: return "ok";
    case HULL_EINVAL: return "invalid argument";
    case HULL_ERANGE: return "coordinate out of range (|x|, |y| must be <= 2^29)";
    case HULL_ENOMEM: return "device memory allocation failed";
    case HULL_ECAPACITY: return "output capacity below the hull size";
    case HULL_ETIMEOUT: return "a bounded device wait timed out";
    case HULL_ECUDA: return "CUDA runtime error";
    case HULL_EINTERNAL: return "internal index check failed";
  }
  return "unknown status";
}

hull_status hull_create(hull_ctx** out, int device, const hull_config* cfg) {
  if (!out) return HULL_EINVAL;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess) return cuda_fail(cudaErrorUnknown);
  if (device < 0 || device >= ndev) return HULL_EINVAL;
  DevGuard g(device);
  hull_ctx* c = new (std::nothrow) hull_ctx();
  if (!c) return HULL_ENOMEM;
  c->device = device;
  if (cfg) c->cfg = *cfg;
  if (c->cfg.spin_limit == 0) c->cfg.spin_limit = kDefaultSpinLimit;
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) { delete c; return cuda_fail(cudaErrorUnknown); }
  c->num_sms = prop.multiProcessorCount;
  if (k2_configure() != cudaSuccess || k3_configure() != cudaSuccess || bucket_configure() != cudaSuccess ||
      fused_configure() != cudaSuccess || fused_occupancy(&c->occ_kf) != cudaSuccess ||
      k1_poly_configure() != cudaSuccess ||
      bucket_occupancy(&c->occ_kb) != cudaSuccess ||
      split_occupancy(&c->occ_sp) != cudaSuccess ||
      k5_configure(&c->occ_k5) != cudaSuccess ||
      k2_occupancy(&c->occ_k2c, &c->occ_k2) != cudaSuccess || k3_occupancy(&c->occ_k3) != cudaSuccess ||
      k4_occupancy(&c->occ_k4) != cudaSuccess) {
    delete c;
    return cuda_fail(cudaErrorUnknown);
  }
  if (c->occ_k5 < 1 || c->occ_kb < 1 || c->occ_sp < 1 || c->occ_kf < 1) {
    delete c;
    return HULL_ECUDA;
  }
  if (batch_configure(&c->occ_b256, &c->occ_b512) != cudaSuccess ||
      seg_configure(&c->occ_sx, &c->occ_sf) != cudaSuccess ||
      cudaStreamCreateWithFlags(&c->aux, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->bev[0], cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->bev[1], cudaEventDisableTiming) != cudaSuccess) {
    delete c;
    return cuda_fail(cudaErrorUnknown);
  }
  if (c->occ_b256 < 1) c->occ_b256 = 1;
  if (c->occ_b512 < 1) c->occ_b512 = 1;
  if (cudaMalloc(&c->plan, sizeof(Plan)) != cudaSuccess) { delete c; return HULL_ENOMEM; }
  if (cudaMemset(c->plan, 0, sizeof(Plan)) != cudaSuccess ||
      cudaMallocHost(&c->h_plan, sizeof(Plan)) != cudaSuccess) {
    cudaFree(c->plan);
    delete c;
    return HULL_ENOMEM;
  }
  std::memset(c->h_plan, 0, sizeof(Plan));
  {
    const size_t np = (size_t)mlp_num_params();
    if (cudaMalloc(&c->W, np * 4) != cudaSuccess || cudaMalloc(&c->W16, np * 2) != cudaSuccess ||
        cudaMalloc(&c->adam_m, np * 4) != cudaSuccess || cudaMalloc(&c->adam_v, np * 4) != cudaSuccess ||
        cudaMalloc(&c->grad, np * 4) != cudaSuccess || cudaMalloc(&c->feat, 64 * 4) != cudaSuccess ||
        cudaMalloc(&c->ext, 32 * 4) != cudaSuccess || cudaMalloc(&c->ext_xy, 64 * 4) != cudaSuccess ||
        cudaMalloc(&c->lab_cnt, 33 * 8) != cudaSuccess || cudaMalloc(&c->d_loss, 16) != cudaSuccess) {
      cudaGetLastError();
      *out = c;
      hull_destroy(c);
      *out = nullptr;
      return HULL_ENOMEM;
    }
    cudaMemset(c->W, 0, np * 4);
    cudaMemset(c->W16, 0, np * 2);
    cudaMemset(c->adam_m, 0, np * 4);
    cudaMemset(c->adam_v, 0, np * 4);
  }
  *out = c;
  return HULL_OK;
}

void hull_destroy(hull_ctx* c) {
  if (!c) return;
  DevGuard g(c->device);
  cudaDeviceSynchronize();
  free_ws(c->ws);
  free_ws(c->ws2);
  if (c->plan2) cudaFree(c->plan2);
  if (c->ang) cudaFree(c->ang);
  if (c->hs.d_in) cudaFree(c->hs.d_in);
  if (c->hs.d_out) cudaFree(c->hs.d_out);
  if (c->hs.d_in2) cudaFree(c->hs.d_in2);
  for (int k = 0; k < 2; ++k) {
    if (c->hs.copied[k]) cudaEventDestroy(c->hs.copied[k]);
    if (c->hs.consumed[k]) cudaEventDestroy(c->hs.consumed[k]);
  }
  if (c->hs.copy) cudaStreamDestroy(c->hs.copy);
  for (int k = 0; k <= HULL_NUM_STAGES; ++k)
    if (c->ev[k]) cudaEventDestroy(c->ev[k]);
  for (void* p : {(void*)c->W, c->W16, (void*)c->adam_m, (void*)c->adam_v, (void*)c->grad, (void*)c->feat,
                  (void*)c->ext, (void*)c->ext_xy, (void*)c->lab_cnt, (void*)c->d_loss, (void*)c->act,
                  (void*)c->scratch})
    if (p) cudaFree(p);
  if (c->bw.base) cudaFree(c->bw.base);
  if (c->bw.slot0) cudaFree(c->bw.slot0);
  if (c->bw.h_off) cudaFreeHost(c->bw.h_off);
  if (c->bw.h_slot0) cudaFreeHost(c->bw.h_slot0);
  if (c->bw.h_order) cudaFreeHost(c->bw.h_order);
  if (c->bw.h_ctl) cudaFreeHost(c->bw.h_ctl);
  if (c->bw.h_tfirst) cudaFreeHost(c->bw.h_tfirst);
  if (c->bw.seg) cudaFree(c->bw.seg);
  for (int k = 0; k < 2; ++k)
    if (c->bev[k]) cudaEventDestroy(c->bev[k]);
  if (c->aux) cudaStreamDestroy(c->aux);
  if (c->plan) cudaFree(c->plan);
  if (c->h_plan) cudaFreeHost(c->h_plan);
  if (c->h_multi) cudaFreeHost(c->h_multi);
  delete c;
}

hull_status hull_compute(hull_ctx* c, const int32_t* d_xy, int64_t n, int32_t* d_out, int64_t cap,
                         int64_t* h_count, void* stream) {
  if (!c || !h_count || n < 0 || cap < 0 || n > (int64_t)kMaxN) return HULL_EINVAL;
  if (n > 0 && (!d_xy || !aligned8(d_xy))) return HULL_EINVAL;
  if (cap > 0 && !d_out) return HULL_EINVAL;
  *h_count = 0;
  if (n == 0) {
    if (c->cfg.collect_stats) c->last = hull_stats{};
    return HULL_OK;
  }
  DevGuard g(c->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  hull_status r = ensure_ws(c, (size_t)n);
  if (r != HULL_OK) return r;
  // The bucket sort first; a bin it cannot sort in shared memory (heavily
  // duplicated or extremely clustered input) reruns the call on the radix
  // passes, which take any input.
  for (int attempt = 0; attempt < 2; ++attempt) {
    const bool bucket = attempt == 0;
    c->prof_pending = c->prof;
    r = run_front(c, d_xy, (u32)n, st, bucket);
    if (r != HULL_OK) { c->prof_pending = false; return r; }
    r = run_final(c, c->ws.lo_xy, c->ws.lo_idx, c->ws.up_xy, c->ws.up_idx, (size_t)n, d_out, cap, st);
    if (r != HULL_OK) c->prof_pending = false;
    if (r != HULL_OK) return r;
    bool fallback = false;
    r = finish(c, st, bucket ? &fallback : nullptr);
    if (fallback) {
      c->fallbacks += 1;
      continue;
    }
    if (c->cfg.collect_stats) c->last.sort_fallback = attempt;
    if (r == HULL_OK || r == HULL_ECAPACITY) *h_count = c->h_plan->h;
    return r;
  }
  return r;
}

hull_status hull_compute_multi(hull_ctx* c, int32_t count, const int32_t* const* d_xy, const int64_t* n,
                               int32_t* const* d_out, const int64_t* cap, int64_t* h_count, void* stream) {
  if (!c || count < 0) return HULL_EINVAL;
  if (count == 0) return HULL_OK;
  if (!d_xy || !n || !d_out || !cap || !h_count) return HULL_EINVAL;
  int64_t nmax = 1;
  for (int32_t k = 0; k < count; ++k) {
    h_count[k] = 0;
    if (n[k] < 0 || cap[k] < 0 || n[k] > (int64_t)kMaxN || (n[k] > 0 && (!d_xy[k] || !aligned8(d_xy[k]))) ||
        (cap[k] > 0 && !d_out[k]))
      return HULL_EINVAL;
    nmax = n[k] > nmax ? n[k] : nmax;
  }
  // Stage events are per call: with profiling on, one call after another.
  if (c->prof) {
    for (int32_t k = 0; k < count; ++k) {
      const hull_status r = hull_compute(c, d_xy[k], n[k], d_out[k], cap[k], &h_count[k], stream);
      if (r != HULL_OK) return r;
    }
    return HULL_OK;
  }
  DevGuard g(c->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  hull_status r = ensure_ws(c, (size_t)nmax);
  if (r != HULL_OK) return r;
  if (c->h_multi_cap < count) {
    if (c->h_multi) cudaFreeHost(c->h_multi);
    c->h_multi = nullptr;
    c->h_multi_cap = 0;
    if (cudaMallocHost(&c->h_multi, (size_t)count * kSummaryBytes) != cudaSuccess) {
      cudaGetLastError();
      return HULL_ENOMEM;
    }
    c->h_multi_cap = count;
  }
  // Two lanes when there are two inputs or more (and no learned proposal,
  // whose buffers are per context): input k runs on lane k % 2, lane 0 on
  // the caller's stream with the context's workspace and Plan, lane 1 on
  // the aux stream with the second ones, so that one hull's latency-bound
  // back half overlaps the other's streaming front.  Every summary is
  // copied to its own slot; one synchronisation.
  const bool two = count >= 2 && !(c->cfg.proposal == 1 && c->have_weights);
  if (two) {
    std::swap(c->ws, c->ws2);
    r = ensure_ws(c, (size_t)nmax);
    std::swap(c->ws, c->ws2);
    if (r != HULL_OK) return r;
    if (!c->plan2) {
      if (cudaMalloc(&c->plan2, sizeof(Plan)) != cudaSuccess) {
        cudaGetLastError();
        return HULL_ENOMEM;
      }
      if (cudaMemsetAsync(c->plan2, 0, sizeof(Plan), st) != cudaSuccess) return cuda_fail(cudaGetLastError());
    }
    cudaError_t e = cudaEventRecord(c->bev[0], st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(c->aux, c->bev[0], 0);
    if (e != cudaSuccess) return cuda_fail(e);
  }
  for (int32_t k = 0; k < count; ++k) {
    if (n[k] == 0) continue;
    const bool lane1 = two && (k & 1);
    const cudaStream_t ls = lane1 ? c->aux : st;
    if (lane1) { std::swap(c->ws, c->ws2); std::swap(c->plan, c->plan2); }
    c->prof_pending = false;
    r = run_front(c, d_xy[k], (u32)n[k], ls, true);
    if (r == HULL_OK) r = run_final(c, c->ws.lo_xy, c->ws.lo_idx, c->ws.up_xy, c->ws.up_idx, (size_t)n[k], d_out[k],
                                    cap[k], ls);
    cudaError_t e = cudaSuccess;
    if (r == HULL_OK)
      e = cudaMemcpyAsync(c->h_multi + (size_t)k * kSummaryBytes, c->plan, kSummaryBytes, cudaMemcpyDeviceToHost, ls);
    if (lane1) { std::swap(c->ws, c->ws2); std::swap(c->plan, c->plan2); }
    if (r != HULL_OK) {
      if (two) cudaStreamSynchronize(c->aux);
      return r;
    }
    if (e != cudaSuccess) return cuda_fail(e);
  }
  if (two) {
    cudaError_t e = cudaEventRecord(c->bev[1], c->aux);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, c->bev[1], 0);
    if (e != cudaSuccess) return cuda_fail(e);
  }
  const cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e);
  hull_status first = HULL_OK;
  for (int32_t k = 0; k < count; ++k) {
    if (n[k] == 0) {
      if (c->cfg.collect_stats) c->last = hull_stats{};
      continue;
    }
    bool fallback = false;
    const Plan& p = *reinterpret_cast<const Plan*>(c->h_multi + (size_t)k * kSummaryBytes);
    r = read_summary(c, p, &fallback);
    if (fallback) {
      // A bin too large for the bucket sort: this input again, as
      // hull_compute does (the radix passes after the bucket attempt).
      r = hull_compute(c, d_xy[k], n[k], d_out[k], cap[k], &h_count[k], stream);
    } else {
      if (c->cfg.collect_stats) c->last.sort_fallback = 0;
      if (r == HULL_OK || r == HULL_ECAPACITY) h_count[k] = p.h;
    }
    if (r != HULL_OK && first == HULL_OK) first = r;
  }
  return first;
}

hull_status hull_stage_sorted_survivors(hull_ctx* c, const int32_t* d_xy, int64_t n, int32_t* d_xy_out,
                                        int32_t* d_idx_out, int64_t cap, int64_t* h_count, void* stream) {
  if (!c || !d_xy || !d_xy_out || !d_idx_out || !h_count || n < 1 || cap < 0 || n > (int64_t)kMaxN || !aligned8(d_xy))
    return HULL_EINVAL;
  *h_count = 0;
  DevGuard g(c->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  hull_status r = ensure_ws(c, (size_t)n);
  if (r != HULL_OK) return r;
  Workspace& w = c->ws;
  cudaError_t e = launch_k1(d_xy, (u32)n, c->cfg.spin_limit, c->plan, w.partials, k1_grid((u32)n, c->num_sms), st);
  if (e != cudaSuccess) return cuda_fail(e);
  const size_t t2 = ((size_t)n + k2_tile() - 1) / k2_tile();
  e = launch_k2(d_xy, c->plan, w.keys[0], w.idx[0], w.st_filter, w.mask, grid_for(c->occ_k2c, c->num_sms, t2),
                grid_for(c->occ_k2, c->num_sms, t2), st);
  const size_t t3 = ((size_t)n + k3_tile() - 1) / k3_tile();
  for (u32 p = 0; e == cudaSuccess && p < (u32)kMaxPasses; ++p)
    e = launch_k3(w.keys[p & 1], w.idx[p & 1], w.keys[(p + 1) & 1], w.idx[(p + 1) & 1], c->plan, w.st_sort, p,
                  grid_for(c->occ_k3, c->num_sms, t3), st);
  if (e == cudaSuccess)
    e = launch_gather_sorted(reinterpret_cast<const int2*>(d_xy), w.idx[0], w.idx[1], c->plan,
                             reinterpret_cast<int2*>(d_xy_out), d_idx_out, (u32)cap, st);
  if (e != cudaSuccess) return cuda_fail(e);
  r = finish(c, st);
  *h_count = c->h_plan->s;
  if (r == HULL_OK && (int64_t)c->h_plan->s > cap) r = HULL_ECAPACITY;
  return r;
}

// The angular variant's scratch: carved in order from the context's
// angular area, which grows (after a device synchronisation) when a call
// needs more and is then kept.  Two carvers may share the area: the
// outer call (hull_compute_angular) carves first and passes its end as the
// inner call's start.
struct AngCarve {
  hull_ctx* c;
  size_t off;
  size_t need = 0;
  bool measure;
  AngCarve(hull_ctx* cc, size_t start, bool m) : c(cc), off(start), measure(m) {}
  void* take(size_t bytes) {
    const size_t o = off;
    off = align_up(off + (bytes < 16 ? 16 : bytes), 256);
    need = off;
    return measure ? nullptr : static_cast<char*>(c->ang) + o;
  }
};

cudaError_t ang_reserve(hull_ctx* c, size_t bytes) {
  if (bytes <= c->ang_bytes && c->ang) return cudaSuccess;
  cudaDeviceSynchronize();
  if (c->ang) cudaFree(c->ang);
  c->ang = nullptr;
  c->ang_bytes = 0;
  const size_t b = align_up(bytes, (size_t)1 << 20);
  const cudaError_t e = cudaMalloc(&c->ang, b);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return e;
  }
  c->ang_bytes = b;
  return cudaSuccess;
}

// Bytes of hull_stage_angular's scratch for n points.
size_t ang_stage_bytes(size_t n) {
  AngCarve m(nullptr, 0, true);
  m.take(n * 4); m.take(n * 8); m.take(n * 4); m.take(n * 8); m.take(n * 4); m.take((n + 1) * 8); m.take(16);
  m.take(angle_walk_scratch_bytes((u32)n + 1));
  return m.need;
}

hull_status ang_stage(hull_ctx* c, const int32_t* d_xy, int64_t n, int32_t* d_order, uint8_t* d_keep,
                      int64_t cap, int64_t* h_m, int64_t* h_l, void* stream, size_t start);

hull_status hull_stage_angular(hull_ctx* c, const int32_t* d_xy, int64_t n, int32_t* d_order, uint8_t* d_keep,
                               int64_t cap, int64_t* h_m, int64_t* h_l, void* stream) {
  if (!c || !d_xy || !h_m || !h_l || n < 1 || cap < 0 || n > (int64_t)kMaxN || !aligned8(d_xy)) return HULL_EINVAL;
  if (cap > 0 && (!d_order || !d_keep)) return HULL_EINVAL;
  *h_m = 0;
  *h_l = -1;
  DevGuard g(c->device);
  if (ang_reserve(c, ang_stage_bytes((size_t)n)) != cudaSuccess) return HULL_ENOMEM;
  return ang_stage(c, d_xy, n, d_order, d_keep, cap, h_m, h_l, stream, 0);
}

hull_status ang_stage(hull_ctx* c, const int32_t* d_xy, int64_t n, int32_t* d_order, uint8_t* d_keep,
                      int64_t cap, int64_t* h_m, int64_t* h_l, void* stream, size_t start) {
  *h_m = 0;
  *h_l = -1;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int32_t ext[4];
  hull_status r = hull_stage_extremes(c, d_xy, n, ext, stream);
  if (r != HULL_OK) return r;
  const u32 anchor = (u32)ext[2];
  const size_t nn = (size_t)n;
  AngCarve t(c, start, false);
  void* keep = t.take(nn * 4);
  void* k1 = t.take(nn * 8);
  void* v1 = t.take(nn * 4);
  void* k2 = t.take(nn * 8);
  void* v2 = t.take(nn * 4);
  void* pts = t.take((nn + 1) * 8);
  void* small = t.take(16);     // [0] points equal to the anchor, [1] P_l's position
  void* walk = t.take(angle_walk_scratch_bytes((u32)n + 1));
  cudaError_t e = cudaSuccess;
  int64_t s = 0;
  r = hull_stage_filter(c, d_xy, n, static_cast<int32_t*>(keep), &s, stream);
  if (r != HULL_OK) return r;
  u32* n_same = static_cast<u32*>(small);
  u32* lpos = n_same + 1;
  const int2* xy2 = reinterpret_cast<const int2*>(d_xy);
  e = cudaMemsetAsync(n_same, 0, 4, st);
  if (e == cudaSuccess)
    e = launch_angle_dist(xy2, static_cast<const int*>(keep), (u32)s, anchor, static_cast<u64*>(k1),
                          static_cast<u32*>(v1), n_same, c->num_sms, st);
  if (e != cudaSuccess) return cuda_fail(e);
  r = hull_stage_sort(c, static_cast<uint64_t*>(k1), static_cast<uint32_t*>(v1), s, stream);
  if (r != HULL_OK) return r;
  e = launch_angle_keys(xy2, static_cast<const u64*>(k1), static_cast<const u32*>(v1), (u32)s, anchor,
                        static_cast<u64*>(k2), static_cast<u32*>(v2), c->num_sms, st);
  if (e != cudaSuccess) return cuda_fail(e);
  r = hull_stage_sort(c, static_cast<uint64_t*>(k2), static_cast<uint32_t*>(v2), s, stream);
  if (r != HULL_OK) return r;
  u32 same = 0;
  e = cudaMemcpyAsync(&same, n_same, 4, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e);
  const int64_t m1 = s - (int64_t)same + 1;
  *h_m = m1;
  if (m1 > cap) return HULL_ECAPACITY;
  e = launch_angle_order(xy2, static_cast<const u32*>(v1), static_cast<const u32*>(v2), (u32)m1, anchor, d_order,
                         static_cast<int2*>(pts), c->num_sms, st);
  if (e != cudaSuccess) return cuda_fail(e);
  if (m1 == 1) {
    e = cudaMemsetAsync(d_keep, 1, 1, st);
  } else {
    e = launch_angle_walks(static_cast<const int2*>(pts), (u32)m1, walk, lpos, d_keep, c->num_sms, st);
    u32 l = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&l, lpos, 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) *h_l = (int64_t)l;
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  return e == cudaSuccess ? HULL_OK : cuda_fail(e);
}

hull_status hull_compute_angular(hull_ctx* c, const int32_t* d_xy, int64_t n, int32_t* d_out, int64_t cap,
                                 int64_t* h_count, void* stream) {
  if (!c || !h_count || n < 0 || cap < 0 || n > (int64_t)kMaxN) return HULL_EINVAL;
  if (n > 0 && (!d_xy || !aligned8(d_xy))) return HULL_EINVAL;
  if (cap > 0 && !d_out) return HULL_EINVAL;
  *h_count = 0;
  if (n == 0) return HULL_OK;
  DevGuard g(c->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t nn = (size_t)n;
  AngCarve m(c, 0, true);
  m.take(nn * 4); m.take(nn + 16); m.take(nn * 4 + 16); m.take(nn * 8); m.take(nn * 4); m.take(nn * 8);
  m.take(nn * 4); m.take(nn * 4);
  if (ang_reserve(c, m.need + ang_stage_bytes(nn)) != cudaSuccess) return HULL_ENOMEM;
  AngCarve t(c, 0, false);
  void* order = t.take(nn * 4);
  void* keep = t.take(nn + 16);
  void* pos = t.take(nn * 4 + 16);      // the count, then the positions
  void* keys = t.take(nn * 8);
  void* vals = t.take(nn * 4);
  void* xyc = t.take(nn * 8);
  void* lab = t.take(nn * 4);
  void* outc = t.take(nn * 4);
  cudaError_t e = cudaSuccess;
  int64_t m1 = 0, l = -1;
  hull_status r = ang_stage(c, d_xy, n, static_cast<int32_t*>(order), static_cast<uint8_t*>(keep), n, &m1, &l,
                            stream, t.off);
  if (r != HULL_OK) return r;
  u32* cnt = static_cast<u32*>(pos);
  u32* ppos = cnt + 4;
  e = cudaMemsetAsync(cnt, 0, 4, st);
  if (e == cudaSuccess)
    e = launch_angle_compact(static_cast<const unsigned char*>(keep), (u32)m1, ppos, cnt, c->num_sms, st);
  u32 rc = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&rc, cnt, 4, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess)
    e = launch_angle_gather(nullptr, nullptr, ppos, rc, static_cast<u64*>(keys), static_cast<u32*>(vals), nullptr,
                            nullptr, c->num_sms, st, 0);
  if (e != cudaSuccess) return cuda_fail(e);
  r = hull_stage_sort(c, static_cast<uint64_t*>(keys), static_cast<uint32_t*>(vals), rc, stream);
  if (r != HULL_OK) return r;
  e = launch_angle_gather(reinterpret_cast<const int2*>(d_xy), static_cast<const int*>(order), ppos, rc,
                          static_cast<u64*>(keys), static_cast<u32*>(vals), static_cast<int2*>(xyc),
                          static_cast<int*>(lab), c->num_sms, st, 1);
  if (e != cudaSuccess) return cuda_fail(e);
  int64_t h = 0;
  r = hull_compute(c, static_cast<const int32_t*>(xyc), rc, static_cast<int32_t*>(outc), rc, &h, stream);
  if (r != HULL_OK) return r;
  *h_count = h;
  if (h > cap) return HULL_ECAPACITY;
  e = launch_angle_label(static_cast<const int*>(outc), static_cast<const int*>(lab), (u32)h, d_out, c->num_sms, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  return e == cudaSuccess ? HULL_OK : cuda_fail(e);
}

hull_status hull_stage_second_round_chunked(hull_ctx* c, const int32_t* d_xy, const int32_t* d_idx, int64_t m,
                                            int32_t block_size, int32_t* d_lower, int64_t* h_lower, int32_t* d_upper,
                                            int64_t* h_upper, void* stream) {
  if (!c || !d_xy || !d_idx || !d_lower || !d_upper || !h_lower || !h_upper || m < 1 || m > (int64_t)kMaxN ||
      !aligned8(d_xy) || block_size < 1 || block_size > 1024)
    return HULL_EINVAL;
  DevGuard g(c->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  hull_status r = ensure_ws(c, (size_t)m);
  if (r != HULL_OK) return r;
  r = new_call_patch(c, st, PlanPatch{});
  if (r != HULL_OK) return r;
  const cudaError_t e = launch_k4_chunked(reinterpret_cast<const int2*>(d_xy), d_idx, (u32)m, (u32)block_size,
                                          c->plan, c->ws.h_idx[0], c->ws.h_idx[1], d_lower, d_upper, st);
  if (e != cudaSuccess) return cuda_fail(e);
  r = finish(c, st);
  *h_lower = c->h_plan->r_lo;
  *h_upper = c->h_plan->r_up;
  return r;
}

hull_status hull_stage_regions(hull_ctx* c, const int32_t* d_xy, int64_t n, int32_t* d_lower,
                               int64_t lower_cap, int32_t* d_upper, int64_t upper_cap, int64_t* h_counts,
                               int32_t* h_fallback, void* stream) {
  if (!c || !h_counts || n < 0 || lower_cap < 0 || upper_cap < 0 || n > (int64_t)kMaxN) return HULL_EINVAL;
  if (n > 0 && (!d_xy || !aligned8(d_xy))) return HULL_EINVAL;
  if ((lower_cap > 0 && !d_lower) || (upper_cap > 0 && !d_upper)) return HULL_EINVAL;
  h_counts[0] = h_counts[1] = 0;
  if (h_fallback) *h_fallback = 0;
  if (n == 0) return HULL_OK;
  DevGuard g(c->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  hull_status r = ensure_ws(c, (size_t)n);
  if (r != HULL_OK) return r;
  for (int attempt = 0; attempt < 2; ++attempt) {
    const bool bucket = attempt == 0;
    c->prof_pending = false;
    r = run_front(c, d_xy, (u32)n, st, bucket, true);   // Figure 2's lists on every first-round survivor
    if (r != HULL_OK) return r;
    bool fallback = false;
    r = finish(c, st, bucket ? &fallback : nullptr);
    if (fallback) continue;
    if (r != HULL_OK) return r;
    if (h_fallback) *h_fallback = attempt;
    const int64_t rl = c->h_plan->r_lo, ru = c->h_plan->r_up;
    h_counts[0] = rl;
    h_counts[1] = ru;
    if (rl > lower_cap || ru > upper_cap) return HULL_ECAPACITY;
    cudaError_t e = cudaSuccess;
    if (rl > 0) e = cudaMemcpyAsync(d_lower, c->ws.lo_idx + 1, (size_t)rl * sizeof(int32_t),
                                    cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess && ru > 0)
      e = cudaMemcpyAsync(d_upper, c->ws.up_idx + 1, (size_t)ru * sizeof(int32_t), cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return e == cudaSuccess ? HULL_OK : cuda_fail(e);
  }
  return r;
}

hull_status hull_compute_host(hull_ctx* c, const int32_t* h_xy, int64_t n, int32_t* h_out,
                              int64_t cap, int64_t* h_count, void* stream) {
  if (!c || !h_count || n < 0 || cap < 0 || n > (int64_t)kMaxN) return HULL_EINVAL;
  if (n > 0 && !h_xy) return HULL_EINVAL;
  if (cap > 0 && !h_out) return HULL_EINVAL;
  *h_count = 0;
  if (n == 0) return HULL_OK;
  DevGuard g(c->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  hull_status gr = ensure_host_stage(c, (size_t)n, false);
  if (gr != HULL_OK) return gr;
  cudaError_t e = cudaMemcpyAsync(c->hs.d_in, h_xy, (size_t)n * 8, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return cuda_fail(e);
  int64_t h = 0;
  hull_status r = hull_compute(c, c->hs.d_in, n, c->hs.d_out, (int64_t)c->hs.cap, &h, stream);
  if (r != HULL_OK) return r;
  *h_count = h;
  if (h > cap) return HULL_ECAPACITY;
  if (h > 0) {
    e = cudaMemcpyAsync(h_out, c->hs.d_out, (size_t)h * 4, cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return cuda_fail(e);
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e);
  }
  return HULL_OK;
}

hull_status hull_compute_host_multi(hull_ctx* c, int32_t count, const int32_t* const* h_xy,
                                    const int64_t* n, int32_t* const* h_out, const int64_t* cap,
                                    int64_t* h_count, void* stream) {
  if (!c || count < 0) return HULL_EINVAL;
  if (count == 0) return HULL_OK;
  if (!h_xy || !n || !h_out || !cap || !h_count) return HULL_EINVAL;
  for (int32_t k = 0; k < count; ++k) {
    h_count[k] = 0;
    if (n[k] < 0 || cap[k] < 0 || n[k] > (int64_t)kMaxN || (n[k] > 0 && !h_xy[k]) || (cap[k] > 0 && !h_out[k]))
      return HULL_EINVAL;
  }
  DevGuard g(c->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int64_t nmax = 1;
  for (int32_t k = 0; k < count; ++k) nmax = n[k] > nmax ? n[k] : nmax;
  hull_status r = ensure_host_stage(c, (size_t)nmax, true);
  if (r != HULL_OK) return r;
  HostStage& hs = c->hs;
  int32_t* buf[2] = {hs.d_in, hs.d_in2};
  // The copy stream starts after everything already queued on `stream`.
  cudaError_t e = cudaEventRecord(hs.consumed[0], st);
  if (e == cudaSuccess) e = cudaEventRecord(hs.consumed[1], st);
  auto issue_copy = [&](int32_t k) -> cudaError_t {
    const int b = k & 1;
    cudaError_t ce = cudaStreamWaitEvent(hs.copy, hs.consumed[b], 0);
    if (ce == cudaSuccess && n[k] > 0)
      ce = cudaMemcpyAsync(buf[b], h_xy[k], (size_t)n[k] * 8, cudaMemcpyHostToDevice, hs.copy);
    if (ce == cudaSuccess) ce = cudaEventRecord(hs.copied[b], hs.copy);
    return ce;
  };
  if (e == cudaSuccess) e = issue_copy(0);
  if (e != cudaSuccess) return cuda_fail(e);
  for (int32_t k = 0; k < count; ++k) {
    const int b = k & 1;
    // Input k + 1 goes into the other buffer once input k - 1 is done with it.
    if (k + 1 < count) {
      e = issue_copy(k + 1);
      if (e != cudaSuccess) return cuda_fail(e);
    }
    e = cudaStreamWaitEvent(st, hs.copied[b], 0);
    if (e != cudaSuccess) return cuda_fail(e);
    int64_t h = 0;
    if (n[k] > 0) r = hull_compute(c, buf[b], n[k], hs.d_out, (int64_t)hs.cap, &h, stream);
    e = cudaEventRecord(hs.consumed[b], st);
    if (r != HULL_OK) {
      cudaStreamSynchronize(hs.copy);
      return r;
    }
    if (e != cudaSuccess) return cuda_fail(e);
    h_count[k] = h;
    if (h > cap[k]) {
      cudaStreamSynchronize(hs.copy);
      return HULL_ECAPACITY;
    }
    if (h > 0) {
      e = cudaMemcpyAsync(h_out[k], hs.d_out, (size_t)h * 4, cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      if (e != cudaSuccess) return cuda_fail(e);
    }
  }
  return HULL_OK;
}

hull_status hull_set_profiling(hull_ctx* c, int enable) {
  if (!c) return HULL_EINVAL;
  DevGuard g(c->device);
  if (enable && !c->ev[0]) {
    for (int k = 0; k <= HULL_NUM_STAGES; ++k)
      if (cudaEventCreate(&c->ev[k]) != cudaSuccess) return cuda_fail(cudaErrorUnknown);
  }
  c->prof = enable != 0;
  c->profile = hull_profile{};
  return HULL_OK;
}

hull_status hull_get_profile(const hull_ctx* c, hull_profile* out) {
  if (!c || !out) return HULL_EINVAL;
  *out = c->profile;
  return HULL_OK;
}

hull_status hull_last_stats(const hull_ctx* c, hull_stats* out) {
  if (!c || !out) return HULL_EINVAL;
  *out = c->last;
  return HULL_OK;
}

hull_status hull_stage_extremes(hull_ctx* c, const int32_t* d_xy, int64_t n, int32_t* h_ext,
                                void* stream) {
  if (!c || !d_xy || !h_ext || n < 1 || n > (int64_t)kMaxN || !aligned8(d_xy)) return HULL_EINVAL;
  DevGuard g(c->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  hull_status r = ensure_ws(c, (size_t)n);
  if (r != HULL_OK) return r;
  cudaError_t e = launch_k1(d_xy, (u32)n, c->cfg.spin_limit, c->plan, c->ws.partials,
                            k1_grid((u32)n, c->num_sms), st);
  if (e != cudaSuccess) return cuda_fail(e);
  r = finish(c, st);
  for (int j = 0; j < 4; ++j) h_ext[j] = c->h_plan->ext_idx[j];
  return r;
}

hull_status hull_stage_filter(hull_ctx* c, const int32_t* d_xy, int64_t n, int32_t* d_keep,
                              int64_t* h_s, void* stream) {
  if (!c || !d_xy || !d_keep || !h_s || n < 1 || n > (int64_t)kMaxN || !aligned8(d_xy)) return HULL_EINVAL;
  DevGuard g(c->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  hull_status r = ensure_ws(c, (size_t)n);
  if (r != HULL_OK) return r;
  cudaError_t e = launch_k1(d_xy, (u32)n, c->cfg.spin_limit, c->plan, c->ws.partials,
                            k1_grid((u32)n, c->num_sms), st);
  if (e != cudaSuccess) return cuda_fail(e);
  const size_t t2 = ((size_t)n + k2_tile() - 1) / k2_tile();
  e = launch_k2(d_xy, c->plan, c->ws.keys[0], c->ws.idx[0], c->ws.st_filter, c->ws.mask,
                grid_for(c->occ_k2c, c->num_sms, t2), grid_for(c->occ_k2, c->num_sms, t2), st);
  if (e != cudaSuccess) return cuda_fail(e);
  r = finish(c, st);
  if (r != HULL_OK) return r;
  *h_s = c->h_plan->s;
  if (c->h_plan->s > 0) {
    e = cudaMemcpyAsync(d_keep, c->ws.idx[0], (size_t)c->h_plan->s * 4, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return cuda_fail(e);
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e);
  }
  return HULL_OK;
}

hull_status hull_stage_sort(hull_ctx* c, uint64_t* d_keys, uint32_t* d_vals, int64_t m, void* stream) {
  if (!c || m < 0 || m > (int64_t)kMaxN) return HULL_EINVAL;
  if (m == 0) return HULL_OK;
  if (!d_keys || !d_vals) return HULL_EINVAL;
  DevGuard g(c->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  hull_status r = ensure_ws(c, (size_t)m);
  if (r != HULL_OK) return r;
  Workspace& w = c->ws;
  cudaError_t e = cudaMemcpyAsync(w.keys[0], d_keys, (size_t)m * 8, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(w.idx[0], d_vals, (size_t)m * 4, cudaMemcpyDeviceToDevice, st);
  if (e != cudaSuccess) return cuda_fail(e);
  PlanPatch p{};
  p.zero_hist = 1; p.set_s = 1; p.s = (u32)m; p.set_npasses = 1; p.npasses = kMaxPasses;
  r = new_call_patch(c, st, p);
  if (r != HULL_OK) return r;
  e = launch_hist(w.keys[0], c->plan, c->num_sms * 2, st);
  if (e != cudaSuccess) return cuda_fail(e);
  const size_t t3 = ((size_t)m + k3_tile() - 1) / k3_tile();
  for (u32 pp = 0; pp < (u32)kMaxPasses; ++pp) {
    e = launch_k3(w.keys[pp & 1], w.idx[pp & 1], w.keys[(pp + 1) & 1], w.idx[(pp + 1) & 1], c->plan,
                  w.st_sort, pp, grid_for(c->occ_k3, c->num_sms, t3), st);
    if (e != cudaSuccess) return cuda_fail(e);
  }
  // kMaxPasses is even: the result is back in buffer 0.
  e = cudaMemcpyAsync(d_keys, w.keys[0], (size_t)m * 8, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_vals, w.idx[0], (size_t)m * 4, cudaMemcpyDeviceToDevice, st);
  if (e != cudaSuccess) return cuda_fail(e);
  return finish(c, st);
}

int64_t hull_bucket_group_cap(void) { return kGroupCap; }

hull_status hull_stage_bucket_sort(hull_ctx* c, uint64_t* d_keys, uint32_t* d_vals, int64_t m,
                                   int32_t* h_fallback, void* stream) {
  if (!c || m < 0 || m > (int64_t)kMaxN) return HULL_EINVAL;
  if (h_fallback) *h_fallback = 0;
  if (m == 0) return HULL_OK;
  if (!d_keys || !d_vals) return HULL_EINVAL;
  DevGuard g(c->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  hull_status r = ensure_ws(c, (size_t)m);
  if (r != HULL_OK) return r;
  Workspace& w = c->ws;
  cudaError_t e = cudaMemcpyAsync(w.keys[1], d_keys, (size_t)m * 8, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(w.idx[1], d_vals, (size_t)m * 4, cudaMemcpyDeviceToDevice, st);
  if (e != cudaSuccess) return cuda_fail(e);
  PlanPatch p{};
  p.set_s = 1; p.s = (u32)m;
  r = new_call_patch(c, st, p);
  if (r != HULL_OK) return r;
  const int grid = std::min(array_hist_grid((u32)m, c->num_sms), (int)w.rows_cap);
  e = launch_array_bins(w.keys[1], w.idx[1], (u32)m, c->plan, w.key_or, w.rows, w.bstart, w.groups, w.keys[0],
                        w.idx[0], grid, st);
  if (e == cudaSuccess)
    e = launch_bucket_sort(w.keys[0], w.idx[0], w.keys[1], w.idx[1], c->plan, w.groups, w.bscratch,
                           c->occ_kb * c->num_sms, st);
  if (e != cudaSuccess) return cuda_fail(e);
  bool fallback = false;
  r = finish(c, st, &fallback);
  if (r != HULL_OK) return r;
  if (fallback) {
    // The input is untouched: sort it on the radix passes instead.
    if (h_fallback) *h_fallback = 1;
    return hull_stage_sort(c, d_keys, d_vals, m, stream);
  }
  e = cudaMemcpyAsync(d_keys, w.keys[1], (size_t)m * 8, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_vals, w.idx[1], (size_t)m * 4, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  return e == cudaSuccess ? HULL_OK : cuda_fail(e);
}

hull_status hull_stage_second_round(hull_ctx* c, const int32_t* d_xy, const int32_t* d_idx, int64_t m,
                                    int32_t* d_lower, int64_t* h_lower, int32_t* d_upper,
                                    int64_t* h_upper, void* stream) {
  if (!c || !d_xy || !d_idx || !d_lower || !d_upper || !h_lower || !h_upper || m < 1 ||
      m > (int64_t)kMaxN || !aligned8(d_xy))
    return HULL_EINVAL;
  DevGuard g(c->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  hull_status r = ensure_ws(c, (size_t)m);
  if (r != HULL_OK) return r;
  Workspace& w = c->ws;
  // K1 on the sorted list gives P_0 (first) and P_l (first of the last run)
  // and the key layout; K2 with no polygon keeps every point in list order.
  cudaError_t e = launch_k1(d_xy, (u32)m, c->cfg.spin_limit, c->plan, w.partials,
                            k1_grid((u32)m, c->num_sms), st);
  if (e != cudaSuccess) return cuda_fail(e);
  PlanPatch p{};
  p.set_ncorner = 1; p.ncorner = 0;
  e = launch_plan_patch(c->plan, p, st);
  if (e != cudaSuccess) return cuda_fail(e);
  const size_t t = ((size_t)m + k2_tile() - 1) / k2_tile();
  e = launch_k2(d_xy, c->plan, w.keys[0], w.idx[0], w.st_filter, w.mask, grid_for(c->occ_k2c, c->num_sms, t),
                grid_for(c->occ_k2, c->num_sms, t), st);
  if (e != cudaSuccess) return cuda_fail(e);
  PlanPatch q{};
  q.set_npasses = 1; q.npasses = 0;
  e = launch_plan_patch(c->plan, q, st);
  if (e != cudaSuccess) return cuda_fail(e);
  const size_t t4 = ((size_t)m + k4_tile() - 1) / k4_tile();
  e = launch_k4(w.keys[0], w.idx[0], w.keys[1], w.idx[1], c->plan, w.st_region, t4, w.lo_xy, w.lo_idx,
                w.up_xy, w.up_idx, w.h_xy[0], w.h_idx[0], w.h_xy[1], w.h_idx[1],
                grid_for(c->occ_k4, c->num_sms, t4), st);
  if (e != cudaSuccess) return cuda_fail(e);
  // The region lists hold list positions at [1, r]; map them to labels.
  e = launch_gather_labels(w.lo_idx, d_idx, &c->plan->r_lo, 1, d_lower, (u32)m, st);
  if (e == cudaSuccess) e = launch_gather_labels(w.up_idx, d_idx, &c->plan->r_up, 1, d_upper, (u32)m, st);
  if (e != cudaSuccess) return cuda_fail(e);
  r = finish(c, st);
  *h_lower = c->h_plan->r_lo;
  *h_upper = c->h_plan->r_up;
  return r;
}

hull_status hull_stage_chain(hull_ctx* c, const int32_t* d_xy, int64_t m, int32_t* d_out, int64_t cap,
                             int64_t* h_lower, int64_t* h_upper, void* stream) {
  if (!c || !d_xy || !h_lower || !h_upper || m < 2 || m > (int64_t)kMaxN / 2 || cap < 0 ||
      (cap > 0 && !d_out) || !aligned8(d_xy))
    return HULL_EINVAL;
  DevGuard g(c->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  hull_status r = ensure_ws(c, (size_t)m * 2);
  if (r != HULL_OK) return r;
  Workspace& w = c->ws;
  cudaError_t e = launch_iota(w.aux, (u32)m, st);
  if (e != cudaSuccess) return cuda_fail(e);
  PlanPatch p{};
  p.set_r = 1; p.r_lo = (u32)m - 2; p.r_up = (u32)m - 2;
  r = new_call_patch(c, st, p);
  if (r != HULL_OK) return r;
  const int2* xy = reinterpret_cast<const int2*>(d_xy);
  r = run_final(c, xy, w.aux, xy, w.aux, (size_t)m * 2, d_out, cap, st);
  if (r != HULL_OK) return r;
  r = finish(c, st);
  *h_lower = c->h_plan->h_lo;
  *h_upper = c->h_plan->h_up;
  return r;
}

// ---------------------------------------------------------------- learned

static uint32_t crc32_bytes(const void* data, size_t len) {
  const unsigned char* p = static_cast<const unsigned char*>(data);
  uint32_t c = 0xFFFFFFFFu;
  for (size_t i = 0; i < len; ++i) {
    c ^= p[i];
    for (int k = 0; k < 8; ++k) c = (c >> 1) ^ (0xEDB88320u & (0u - (c & 1u)));
  }
  return ~c;
}

int64_t hull_mlp_num_params(void) { return mlp_num_params(); }

hull_status hull_mlp_set_params(hull_ctx* c, const float* h_params, int64_t count) {
  if (!c || !h_params || count != mlp_num_params()) return HULL_EINVAL;
  DevGuard g(c->device);
  cudaError_t e = cudaMemcpy(c->W, h_params, (size_t)count * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = launch_to_half(c->W, c->W16, (int)count, nullptr);
  if (e == cudaSuccess) e = cudaMemset(c->adam_m, 0, (size_t)count * 4);
  if (e == cudaSuccess) e = cudaMemset(c->adam_v, 0, (size_t)count * 4);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(e);
  c->adam_step = 0;
  c->have_weights = true;
  return HULL_OK;
}

hull_status hull_mlp_get_params(const hull_ctx* c, float* h_params, int64_t count) {
  if (!c || !h_params || count != mlp_num_params()) return HULL_EINVAL;
  DevGuard g(c->device);
  cudaError_t e = cudaMemcpy(h_params, c->W, (size_t)count * 4, cudaMemcpyDeviceToHost);
  return e == cudaSuccess ? HULL_OK : cuda_fail(e);
}

hull_status hull_save_proposal(const hull_ctx* c, const char* path) {
  if (!c || !path) return HULL_EINVAL;
  const int64_t np = mlp_num_params();
  std::vector<float> w((size_t)np);
  hull_status r = hull_mlp_get_params(c, w.data(), np);
  if (r != HULL_OK) return r;
  FILE* f = std::fopen(path, "wb");
  if (!f) return HULL_EINVAL;
  const uint32_t hdr[8] = {0x4C484247u /* "GBHL" */, 1u, 64u, 128u, 128u, 32u, (uint32_t)np,
                           crc32_bytes(w.data(), w.size() * 4)};
  const bool ok = std::fwrite(hdr, 4, 8, f) == 8 && std::fwrite(w.data(), 4, w.size(), f) == w.size();
  std::fclose(f);
  return ok ? HULL_OK : HULL_EINVAL;
}

hull_status hull_load_proposal(hull_ctx* c, const char* path) {
  if (!c || !path) return HULL_EINVAL;
  FILE* f = std::fopen(path, "rb");
  if (!f) return HULL_EINVAL;
  uint32_t hdr[8];
  const int64_t np = mlp_num_params();
  std::vector<float> w((size_t)np);
  const bool ok = std::fread(hdr, 4, 8, f) == 8 && hdr[0] == 0x4C484247u && hdr[1] == 1u && hdr[2] == 64u &&
                  hdr[3] == 128u && hdr[4] == 128u && hdr[5] == 32u && hdr[6] == (uint32_t)np &&
                  std::fread(w.data(), 4, w.size(), f) == w.size();
  std::fclose(f);
  if (!ok || crc32_bytes(w.data(), w.size() * 4) != hdr[7]) return HULL_EINVAL;
  return hull_mlp_set_params(c, w.data(), np);
}

hull_status hull_learned_features(hull_ctx* c, const int32_t* d_xy, int64_t n, float* d_feat,
                                  int32_t* d_ext, int32_t* d_ext_xy, void* stream) {
  if (!c || !d_xy || n < 1 || n > (int64_t)kMaxN || !aligned8(d_xy) || !d_feat || !d_ext || !d_ext_xy)
    return HULL_EINVAL;
  DevGuard g(c->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e = launch_features(d_xy, (u32)n, d_feat, d_ext, d_ext_xy, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  return e == cudaSuccess ? HULL_OK : cuda_fail(e);
}

hull_status hull_learned_labels(hull_ctx* c, const int32_t* d_xy, int64_t n, float* h_labels,
                                float* h_quad_frac, void* stream) {
  if (!c || !d_xy || n < 1 || n > (int64_t)kMaxN || !aligned8(d_xy) || !h_labels) return HULL_EINVAL;
  DevGuard g(c->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  hull_status r = ensure_ws(c, (size_t)n);
  if (r != HULL_OK) return r;
  // Quadrilateral from K1, the 32 extremes from K6, then exact counts.
  cudaError_t e = launch_k1(d_xy, (u32)n, c->cfg.spin_limit, c->plan, c->ws.partials,
                            k1_grid((u32)n, c->num_sms), st);
  if (e == cudaSuccess) e = launch_features(d_xy, (u32)n, c->feat, c->ext, c->ext_xy, st);
  if (e != cudaSuccess) return cuda_fail(e);
  r = finish(c, st);
  if (r != HULL_OK) return r;
  int quad[8];
  const int nq = c->h_plan->ncorner;
  for (int j = 0; j < nq && j < 4; ++j) { quad[2 * j] = c->h_plan->cx[j]; quad[2 * j + 1] = c->h_plan->cy[j]; }
  int* d_quad = c->ws.aux;
  e = cudaMemcpyAsync(d_quad, quad, sizeof(quad), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->lab_cnt, 0, 33 * 8, st);
  if (e == cudaSuccess) e = launch_labels(d_xy, (u32)n, d_quad, nq, c->ext_xy, c->lab_cnt, c->num_sms * 4, st);
  unsigned long long cnt[33];
  if (e == cudaSuccess) e = cudaMemcpyAsync(cnt, c->lab_cnt, sizeof(cnt), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e);
  for (int j = 0; j < 32; ++j) h_labels[j] = (float)((double)((long long)cnt[j] - (long long)cnt[32]) / (double)n);
  if (h_quad_frac) *h_quad_frac = (float)((double)cnt[32] / (double)n);
  return HULL_OK;
}

static hull_status ensure_train(hull_ctx* c, int B) {
  if ((size_t)B <= c->train_cap) return HULL_OK;
  if (c->act) cudaFree(c->act);
  if (c->scratch) cudaFree(c->scratch);
  c->act = nullptr; c->scratch = nullptr; c->train_cap = 0;
  const size_t rows = (size_t)B;
  if (cudaMalloc(&c->act, rows * (128 + 128 + 32) * 4) != cudaSuccess ||
      cudaMalloc(&c->scratch, rows * (128 + 128 + 32) * 4) != cudaSuccess) {
    cudaGetLastError();
    return HULL_ENOMEM;
  }
  c->train_cap = rows;
  return HULL_OK;
}

hull_status hull_mlp_forward(hull_ctx* c, const float* d_X, int32_t B, float* d_Z, void* stream) {
  if (!c || !d_X || !d_Z || B < 1) return HULL_EINVAL;
  DevGuard g(c->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  hull_status r = ensure_train(c, B);
  if (r != HULL_OK) return r;
  cudaError_t e = mlp_forward(c->W, d_X, B, c->act, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d_Z, c->act + (size_t)B * 256, (size_t)B * 32 * 4, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  return e == cudaSuccess ? HULL_OK : cuda_fail(e);
}

hull_status hull_mlp_gradient(hull_ctx* c, const float* d_X, const float* d_Y, int32_t B, float* h_grad,
                              float* h_loss, void* stream) {
  if (!c || !d_X || !d_Y || B < 1) return HULL_EINVAL;
  DevGuard g(c->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  hull_status r = ensure_train(c, B);
  if (r != HULL_OK) return r;
  cudaError_t e = mlp_forward(c->W, d_X, B, c->act, st);
  if (e == cudaSuccess) e = mlp_backward(c->W, d_X, d_Y, B, c->act, c->grad, c->d_loss, c->scratch, st);
  if (e == cudaSuccess && h_grad)
    e = cudaMemcpyAsync(h_grad, c->grad, (size_t)mlp_num_params() * 4, cudaMemcpyDeviceToHost, st);
  float loss = 0.f;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&loss, c->d_loss, 4, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e);
  if (h_loss) *h_loss = loss;
  return HULL_OK;
}

hull_status hull_mlp_train_step(hull_ctx* c, const float* d_X, const float* d_Y, int32_t B, float lr,
                                float* h_loss, void* stream) {
  if (!c || !d_X || !d_Y || B < 1 || !(lr > 0.f)) return HULL_EINVAL;
  DevGuard g(c->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  hull_status r = ensure_train(c, B);
  if (r != HULL_OK) return r;
  cudaError_t e = mlp_forward(c->W, d_X, B, c->act, st);
  if (e == cudaSuccess) e = mlp_backward(c->W, d_X, d_Y, B, c->act, c->grad, c->d_loss, c->scratch, st);
  if (e == cudaSuccess) e = mlp_adam(c->W, c->grad, c->adam_m, c->adam_v, c->adam_step + 1, lr, c->W16, st);
  float loss = 0.f;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&loss, c->d_loss, 4, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e);
  c->adam_step += 1;
  c->have_weights = true;
  if (h_loss) *h_loss = loss;
  return HULL_OK;
}

int64_t hull_batched_max_instance(void) { return (int64_t)batch_max_instance(); }

hull_status hull_compute_batched(hull_ctx* c, const int32_t* d_xy, const int64_t* d_offsets, int32_t B,
                                 int32_t* d_out, int64_t cap, int64_t* d_out_offsets, void* stream) {
  if (!c || B < 0 || cap < 0 || !d_offsets || !d_out_offsets || (cap > 0 && !d_out)) return HULL_EINVAL;
  DevGuard g(c->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  BatchWs& w = c->bw;
  if ((size_t)B + 1 > w.h_cap) {
    if (w.h_off) cudaFreeHost(w.h_off);
    if (w.h_slot0) cudaFreeHost(w.h_slot0);
    if (w.h_order) cudaFreeHost(w.h_order);
    if (w.h_ctl) cudaFreeHost(w.h_ctl);
    if (w.h_tfirst) cudaFreeHost(w.h_tfirst);
    w.h_off = nullptr; w.h_slot0 = nullptr; w.h_order = nullptr; w.h_ctl = nullptr; w.h_tfirst = nullptr;
    w.h_cap = 0;
    const size_t hc = (size_t)B + 1024;
    if (cudaMallocHost(&w.h_off, hc * 8) != cudaSuccess || cudaMallocHost(&w.h_slot0, hc * 8) != cudaSuccess ||
        cudaMallocHost(&w.h_order, hc * 4) != cudaSuccess || cudaMallocHost(&w.h_ctl, 64) != cudaSuccess ||
        cudaMallocHost(&w.h_tfirst, hc * 4) != cudaSuccess) {
      cudaGetLastError();
      return HULL_ENOMEM;
    }
    w.h_cap = hc;
  }
  cudaError_t e = cudaMemcpyAsync(w.h_off, d_offsets, ((size_t)B + 1) * 8, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e);
  if (w.h_off[0] != 0) return HULL_EINVAL;
  const int64_t maxi = (int64_t)batch_max_instance();
  const int64_t pad = batch_pad();
  const int64_t tile = seg_tile();
  int64_t slots = 0, tiles_all = 0;
  for (int i = 0; i < B; ++i) {
    const int64_t ni = w.h_off[i + 1] - w.h_off[i];
    if (ni < 0 || ni > maxi || w.h_off[i + 1] > (int64_t)kMaxN) return HULL_EINVAL;
    w.h_slot0[i] = slots;
    slots += ni + pad;
    tiles_all += (ni + tile - 1) / tile;
  }
  if (B == 0) {
    long long zero = 0;
    e = cudaMemcpyAsync(d_out_offsets, &zero, 8, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return e == cudaSuccess ? HULL_OK : cuda_fail(e);
  }
  if (!d_xy) return HULL_EINVAL;
  // Workspace.
  if ((size_t)slots > w.cap_slots || (size_t)B > w.cap_b) {
    cudaDeviceSynchronize();
    if (w.base) cudaFree(w.base);
    if (w.slot0) cudaFree(w.slot0);
    w.base = nullptr; w.slot0 = nullptr; w.cap_slots = 0; w.cap_b = 0;
    const size_t cs = std::max<size_t>((size_t)slots, (size_t)1 << 20);
    const size_t bytes = cs * (8 + 8 + 4 + 4 + 8 + 4 + 8 + 4 + 4);
    const size_t cb = (size_t)B + 1024;
    if (cudaMalloc(&w.base, bytes) != cudaSuccess ||
        cudaMalloc(&w.slot0, cb * 8 + cb * 4 + cb * 4 + 256) != cudaSuccess) {
      cudaGetLastError();
      if (w.base) cudaFree(w.base);
      w.base = nullptr;
      return HULL_ENOMEM;
    }
    char* b = static_cast<char*>(w.base);
    w.ka = reinterpret_cast<u64*>(b); b += cs * 8;
    w.kb = reinterpret_cast<u64*>(b); b += cs * 8;
    w.lxy = reinterpret_cast<int2*>(b); b += cs * 8;
    w.uxy = reinterpret_cast<int2*>(b); b += cs * 8;
    w.ia = reinterpret_cast<u32*>(b); b += cs * 4;
    w.ib = reinterpret_cast<u32*>(b); b += cs * 4;
    w.lidx = reinterpret_cast<int*>(b); b += cs * 4;
    w.uidx = reinterpret_cast<int*>(b); b += cs * 4;
    w.out_tmp = reinterpret_cast<int*>(b);
    char* t = reinterpret_cast<char*>(w.slot0);
    w.order = reinterpret_cast<int*>(t + cb * 8);
    w.hcount = reinterpret_cast<u32*>(t + cb * 8 + cb * 4);
    w.ctl = reinterpret_cast<u32*>(t + cb * 16);
    w.cap_slots = cs;
    w.cap_b = (size_t)B;
  }
  // Segmented path: room for every instance's tiles and record, whatever
  // the boundary.
  if ((size_t)tiles_all > w.cap_tiles || (size_t)B > w.cap_seg) {
    cudaDeviceSynchronize();
    if (w.seg) cudaFree(w.seg);
    w.seg = nullptr; w.cap_tiles = 0; w.cap_seg = 0;
    const size_t ct = (size_t)tiles_all + 1024, cb = (size_t)B + 1024;
    const size_t b_text = align_up(ct * seg_text_bytes(), 256), b_tcnt = align_up(ct * 4, 256);
    const size_t b_rec = align_up(cb * seg_rec_bytes(), 256), b_tf = align_up((cb + 1) * 4, 256);
    if (cudaMalloc(&w.seg, b_text + b_tcnt + b_rec + b_tf) != cudaSuccess) {
      cudaGetLastError();
      w.seg = nullptr;
      return HULL_ENOMEM;
    }
    char* b = static_cast<char*>(w.seg);
    w.text = b; b += b_text;
    w.tcnt = reinterpret_cast<u32*>(b); b += b_tcnt;
    w.rec = b; b += b_rec;
    w.tfirst = reinterpret_cast<int*>(b);
    w.cap_tiles = (size_t)tiles_all;
    w.cap_seg = (size_t)B;
  }
  e = cudaMemcpyAsync(w.slot0, w.h_slot0, (size_t)B * 8, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return cuda_fail(e);

  // Size buckets: the segmented path (seg_min points or more), large
  // (more than kSmallInstance) and small instances; `order` lists them in
  // that order, each bucket largest first.  The host arrays are rewritten
  // only after the stream has finished the copies of the previous layout.
  int nh = 0, nl = 0, ns = 0, ntiles = 0;
  auto layout = [&](int64_t seg_min) -> cudaError_t {
    cudaError_t r = cudaStreamSynchronize(st);
    if (r != cudaSuccess) return r;
    std::vector<int> huge, large, small;
    for (int i = 0; i < B; ++i) {
      const int64_t ni = w.h_off[i + 1] - w.h_off[i];
      (ni >= seg_min ? huge : ni <= kSmallInstance ? small : large).push_back(i);
    }
    auto by_size = [&](int a, int b) {
      const int64_t na = w.h_off[a + 1] - w.h_off[a], nb = w.h_off[b + 1] - w.h_off[b];
      return na != nb ? na > nb : a < b;
    };
    std::sort(huge.begin(), huge.end(), by_size);
    std::sort(large.begin(), large.end(), by_size);
    std::sort(small.begin(), small.end(), by_size);
    std::copy(huge.begin(), huge.end(), w.h_order);
    std::copy(large.begin(), large.end(), w.h_order + huge.size());
    std::copy(small.begin(), small.end(), w.h_order + huge.size() + large.size());
    nh = (int)huge.size(); nl = (int)large.size(); ns = (int)small.size();
    ntiles = 0;
    for (int h = 0; h < nh; ++h) {
      w.h_tfirst[h] = ntiles;
      ntiles += (int)((w.h_off[huge[h] + 1] - w.h_off[huge[h]] + tile - 1) / tile);
    }
    w.h_tfirst[nh] = ntiles;
    r = cudaMemcpyAsync(w.order, w.h_order, (size_t)B * 4, cudaMemcpyHostToDevice, st);
    if (r == cudaSuccess) r = cudaMemcpyAsync(w.tfirst, w.h_tfirst, ((size_t)nh + 1) * 4, cudaMemcpyHostToDevice, st);
    return r;
  };

  BatchLaunch L{};
  L.xy = d_xy; L.offsets = reinterpret_cast<const long long*>(d_offsets);
  L.slot0 = w.slot0; L.ka = w.ka; L.kb = w.kb; L.ia = w.ia; L.ib = w.ib;
  L.lxy = w.lxy; L.lidx = w.lidx; L.uxy = w.uxy; L.uidx = w.uidx;
  L.out_tmp = w.out_tmp; L.hcount = w.hcount; L.error = w.ctl + 2;
  L.w16 = (c->cfg.proposal == 1 && c->have_weights) ? c->W16 : nullptr;
  L.tfirst = w.tfirst; L.text = w.text; L.tcnt = w.tcnt; L.rec = w.rec;
  // bucket 0 small, 1 large (one block per instance), 2 segmented (the
  // streaming passes over all tiles, plans, the second pass, the gathers)
  // front (bucket 2 only): 1 the streaming passes and the plans, 0 the
  // gathers and back halves, -1 both.
  auto run_bucket = [&](int bucket, int block, cudaStream_t s2, int front = -1) -> cudaError_t {
    BatchLaunch M = L;
    const int occ = block == 512 ? c->occ_b512 : c->occ_b256;
    if (bucket == 2) {
      M.order = w.order;
      M.nb = nh;
      const int grid = std::max(1, std::min(nh, occ * c->num_sms));
      cudaError_t r = cudaSuccess;
      if (front != 0) {
        r = launch_seg_ext(M, ntiles, c->occ_sx * c->num_sms, s2);
        M.mode = 1; M.queue = w.ctl + 3;
        if (r == cudaSuccess) r = launch_batch(block, grid, M, s2);
        if (r == cudaSuccess) r = launch_seg_filter(M, ntiles, c->occ_sf * c->num_sms, s2);
      }
      M.mode = 2; M.queue = w.ctl + 4;
      if (r == cudaSuccess && front != 1) r = launch_batch(block, grid, M, s2);
      return r;
    }
    M.order = w.order + nh + (bucket == 1 ? 0 : nl);
    M.nb = bucket == 1 ? nl : ns;
    M.queue = w.ctl + bucket;
    const int grid = std::max(1, std::min(M.nb, occ * c->num_sms));
    return launch_batch(block, grid, M, s2);
  };
  auto block_of = [&](int bucket) { return c->tuned_block[bucket] ? c->tuned_block[bucket] : 256; };
  // The whole batch.  The segmented bucket's streaming passes run alone on
  // the caller's stream (the one-block kernels are persistent: started
  // beside them they would hold the SMs until their queues drain); then its
  // gathers and back halves run there while the large and then the small
  // instances run on the context's second stream, so that the back halves
  // (latency) share the SMs with those instances' streaming.
  auto run_all = [&]() -> cudaError_t {
    cudaError_t r = cudaMemsetAsync(w.ctl, 0, 64, st);
    if (r == cudaSuccess && nh > 0) r = run_bucket(2, block_of(2), st, 1);
    if (r == cudaSuccess) r = cudaEventRecord(c->bev[0], st);
    if (r == cudaSuccess) r = cudaStreamWaitEvent(c->aux, c->bev[0], 0);
    if (r == cudaSuccess && nh > 0) r = run_bucket(2, block_of(2), st, 0);
    if (r == cudaSuccess && nl > 0) r = run_bucket(1, block_of(1), c->aux);
    if (r == cudaSuccess && ns > 0) r = run_bucket(0, block_of(0), c->aux);
    if (r == cudaSuccess) r = cudaEventRecord(c->bev[1], c->aux);
    if (r == cudaSuccess) r = cudaStreamWaitEvent(st, c->bev[1], 0);
    return r;
  };
  auto timed = [&](auto&& fn) -> float {
    // One warm-up round, then the best of two timed rounds.
    cudaEvent_t t0, t1;
    cudaEventCreate(&t0);
    cudaEventCreate(&t1);
    float best = 1e30f;
    for (int rep = 0; rep < 3; ++rep) {
      cudaEventRecord(t0, st);
      fn();
      cudaEventRecord(t1, st);
      cudaEventSynchronize(t1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, t0, t1);
      if (rep >= 1 && ms < best) best = ms;
    }
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    return best;
  };
  // Autotuning on the first batch: the block size per bucket (each bucket
  // timed alone at the default boundary), then the segmented path's
  // boundary (the whole batch timed at each candidate).
  // The boundary: the caller's (hull_config.batched_seg_min), else the
  // tuned one, else the default.
  const int64_t fixed_seg = c->cfg.batched_seg_min > 0 ? (int64_t)c->cfg.batched_seg_min : 0;
  auto seg_boundary = [&]() { return fixed_seg ? fixed_seg : (c->tuned_seg ? c->tuned_seg : kSegDefault); };
  if (c->cfg.autotune && (c->tuned_block[0] == 0 || c->tuned_block[1] == 0 || c->tuned_block[2] == 0 ||
                          (c->tuned_seg == 0 && !fixed_seg))) {
    autotune_load(c);
    e = layout(seg_boundary());
    if (e != cudaSuccess) return cuda_fail(e);
    for (int bucket = 0; bucket < 3; ++bucket) {
      if (c->tuned_block[bucket] != 0) continue;
      if ((bucket == 0 ? ns : bucket == 1 ? nl : nh) == 0) continue;
      float best = 1e30f;
      int best_b = 256;
      for (int blk : {256, 512}) {
        const float ms = timed([&] {
          cudaMemsetAsync(w.ctl, 0, 64, st);
          run_bucket(bucket, blk, st);
        });
        if (ms < best) { best = ms; best_b = blk; }
      }
      c->tuned_block[bucket] = best_b;
    }
    if (c->tuned_seg == 0 && !fixed_seg) {
      float best = 1e30f;
      int64_t best_t = kSegDefault;
      const int64_t cands[5] = {kSegDefault, kSegCandidates[0], kSegCandidates[1], kSegCandidates[2],
                                kSegCandidates[3]};
      for (int64_t tc : cands) {
        e = layout(tc);
        if (e != cudaSuccess) return cuda_fail(e);
        const float ms = timed(run_all);
        if (ms < best) { best = ms; best_t = tc; }
      }
      c->tuned_seg = best_t;
    }
    autotune_save(c);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e);
  }
  e = layout(seg_boundary());
  if (e == cudaSuccess) e = run_all();
  if (e == cudaSuccess)
    e = launch_batch_output(w.hcount, w.slot0, w.out_tmp, B, reinterpret_cast<long long*>(d_out_offsets),
                            d_out, (long long)cap, w.ctl + 2, c->num_sms * 4, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(w.h_ctl, w.ctl, 16, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e);
  const u32 err = w.h_ctl[2];
  if (err & ERR_RANGE) return HULL_ERANGE;
  if (err & ERR_INTERNAL) return HULL_EINTERNAL;
  if (err & ERR_CAPACITY) return HULL_ECAPACITY;
  return HULL_OK;
}

}  // extern "C"
