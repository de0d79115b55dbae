/*
 * gbhull -- exact 2D convex hull on NVIDIA GB300 (sm_103a).
 *
 * C ABI of the data-parallel hot path of the gScan method (Mei, "gScan:
 * Accelerating Graham Scan on the GPU", arXiv 1508.05931): extreme points
 * (Section 2.1 step 1), quadrilateral filter (step 2, Section 3.1), sort
 * (step 4, Section 3.3), region split and second-round filter (steps 5-7,
 * Section 2.2, Figure 2, Section 3.4) and the finalisation (step 8), every
 * step on the GPU.  The paper's own angular ordering (steps 3-8 with the sort
 * by angle, Sections 3.2-3.3) is available beside it: hull_stage_angular,
 * hull_compute_angular.
 *
 * Conventions shared by every entry point
 *   - Points are int32 (x, y) pairs, array-of-structures, 8 bytes per point,
 *     8-byte aligned (16-byte alignment enables 128-bit loads); every
 *     coordinate must satisfy |x|, |y| <= 2^29, else HULL_ERANGE.
 *   - Orientation tests are exact int64 cross products.
 *   - A hull is the list of its strict vertices (collinear boundary points
 *     excluded) as 0-based input indices, counter-clockwise, starting at the
 *     lexicographically smallest (x, y); among equal points the smallest
 *     index is reported (hull_compute_angular: the first in angular order
 *     among the points its second round keeps; its backward walk keeps the
 *     largest index of equal points).  n = 0 gives 0
 *     vertices, one distinct point gives 1, collinear points give the 2
 *     endpoints.
 *   - Pointers named d_* are device pointers, h_* host pointers.  The
 *     caller owns every buffer it passes; the library never frees or keeps
 *     them past the call.  A context owns its device workspace (grown on
 *     demand, freed by hull_destroy).
 *   - stream is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Work is stream-ordered; calls that return a count to the
 *     host synchronise that stream before returning.
 *   - Errors never trap the GPU and leave no sticky CUDA error: device
 *     waits are bounded and report HULL_ETIMEOUT; every device write is
 *     bounds-checked.  A context is not thread-safe: use one per host
 *     thread (or serialise calls).
 */
#ifndef GBHULL_H
#define GBHULL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hull_ctx hull_ctx;

typedef enum {
  HULL_OK = 0,
  HULL_EINVAL = 1,     /* null/negative/misaligned argument, n >= 2^30 */
  HULL_ERANGE = 2,     /* a coordinate beyond +-2^29; outputs untouched */
  HULL_ENOMEM = 3,     /* workspace allocation failed */
  HULL_ECAPACITY = 4,  /* output capacity below the hull size; count still reported */
  HULL_ETIMEOUT = 5,   /* a bounded device wait ran out; results invalid */
  HULL_ECUDA = 6,      /* a CUDA runtime call failed */
  HULL_EINTERNAL = 7   /* a device index left its buffer (write skipped) */
} hull_status;

typedef struct {
  int proposal;       /* 0 = quadrilateral of the four extremes (the paper), 1 = learned
                         (on the two-read front and in batched mode; the single-read
                         front's sample polygon and witness test leave it nothing to gain) */
  int collect_stats;  /* 1 = keep survivor counts of the last call for hull_last_stats */
  uint32_t spin_limit;/* iteration limit of every device wait; 0 = default (1 << 22) */
  int autotune;       /* 1 = time the batched kernels' block sizes per size bucket and the
                         boundary of the segmented path on first use and cache the choice
                         (file: $GBHULL_AUTOTUNE_CACHE, else ~/.cache/gbhull_autotune.json);
                         0 = built-in defaults */
  int reverse_round;  /* 1 = after the second round (Section 2.2, Figure 2) run it mirrored
                         over each region's survivors -- walked from P_maxx back to P_minx
                         with P_minx as the anchor -- before the final chain (hull_compute,
                         hull_compute_multi, hull_compute_host*, hull_stage_regions; the
                         hull is the same, r_lower / r_upper count the points it keeps);
                         0 = the paper's single second round */
  int batched_seg_min;/* hull_compute_batched: instances of at least this many points take
                         the segmented path (streaming passes over all their tiles at once);
                         0 = the autotuned boundary (autotune = 1) or 65,536; above
                         hull_batched_max_instance(): no instance takes it */
} hull_config;

typedef struct {
  int64_t n;          /* input points */
  int64_t s;          /* survivors of the first-round filter (Section 3.1) */
  int64_t r_lower;    /* second-round survivors, region right of P_minx -> P_maxx */
  int64_t r_upper;    /* second-round survivors, region left of it (Section 2.2) */
  int64_t h;          /* hull vertices */
  int32_t ext[4];     /* indices of P_minx, P_maxx, P_miny, P_maxy (Section 2.1 step 1) */
  int32_t ncorner;    /* distinct corners of the filter polygon */
  int32_t learned_used; /* 1 when the learned polygon replaced the quadrilateral (set on
                           every single-hull call, also without collect_stats) */
  int32_t sort_fallback; /* 1 when the bucket sort met a bin it cannot sort in shared memory
                            and the call was rerun on the radix passes */
  int64_t s_witness;  /* first-round survivors left by the fused filter's test against the
                         sampled witnesses (Figure 2's test against a sampled earlier
                         survivor of the same bin range and region; every point it removes
                         Figure 2 removes too); equals s on the radix passes */
} hull_stats;

/* Creates a context on CUDA device `device` (cfg NULL = defaults).
 * *out receives the context; NULL on failure.  Errors: EINVAL, ECUDA. */
hull_status hull_create(hull_ctx **out, int device, const hull_config *cfg);

/* Frees the context and its workspace.  NULL-safe.  Synchronises the device
 * work the context launched. */
void hull_destroy(hull_ctx *ctx);

/* Convex hull of n points (Section 1's problem; the gScan pipeline of
 * Section 2.1).  d_xy: device int32[n][2], read-only.  d_out: device
 * int32[cap] receiving the CCW vertex indices.  *h_count (host) receives the
 * hull size on HULL_OK and on HULL_ECAPACITY (then d_out is untouched).
 * Synchronises `stream` before returning.  n must be < 2^30.  Inputs of
 * 65,536 points or more, 16-byte aligned, in a context without
 * collect_stats take the single-read front (one pass over the input after a
 * sample polygon drops the points strictly inside a polygon spanned by
 * sampled input points); the others the two-read front (the extremes pass,
 * then the filter pass over the input).  The survivors are sorted by the
 * bucket sort (hull_stage_bucket_sort); an input it cannot handle in shared
 * memory is rerun on the radix passes (hull_stats.sort_fallback), with the
 * same result. */
hull_status hull_compute(hull_ctx *ctx, const int32_t *d_xy, int64_t n, int32_t *d_out,
                         int64_t cap, int64_t *h_count, void *stream);

/* The same computation on host buffers: copies h_xy (n points, preferably
 * pinned) to the device, computes, and copies the vertex indices back into
 * h_out (host int32[cap]).  Same errors as hull_compute. */
hull_status hull_compute_host(hull_ctx *ctx, const int32_t *h_xy, int64_t n, int32_t *h_out,
                              int64_t cap, int64_t *h_count, void *stream);

/* Several independent hulls from device buffers in one call: for k in
 * [0, count), d_xy[k] (device int32[n[k]][2], 8-byte aligned) and d_out[k]
 * (device int32[cap[k]]) as in hull_compute; h_count[k] receives the hull
 * size.  With two inputs or more (and no learned proposal) the inputs
 * alternate between two lanes that run concurrently: even inputs on
 * `stream`, odd ones on an internal stream that first waits for the work
 * queued on `stream` before the call; each lane has its own workspace (the
 * second is allocated by the first such call and kept).  One
 * synchronisation at the end, after both lanes (an input whose bucket sort
 * needs the radix passes is rerun afterwards, alone).  With a single input
 * or the learned proposal, the hulls run back to back on `stream`.
 * Returns the first failing input's status (every
 * other input is still computed; h_count as hull_compute sets it).  With
 * profiling on (hull_set_profiling) the inputs run one call at a time.
 * count = 0 does nothing.  Errors: those of hull_compute; EINVAL for
 * count < 0 or NULL arrays. */
hull_status hull_compute_multi(hull_ctx *ctx, int32_t count, const int32_t *const *d_xy,
                               const int64_t *n, int32_t *const *d_out, const int64_t *cap,
                               int64_t *h_count, void *stream);

/* Several independent hulls from host buffers in one call, pipelined: while
 * the hull of input k is computed on `stream`, input k + 1 is copied to a
 * second device staging buffer on the context's copy stream (inputs should
 * be pinned for the copies to overlap).  For k in [0, count): h_xy[k] holds
 * n[k] points (host int32[n[k]][2]); h_out[k] (host int32[cap[k]]) receives
 * the CCW vertex indices and h_count[k] the hull size.  Stops at the first
 * failing input and returns its status (its h_count is set as by
 * hull_compute_host; later entries are set to 0).  count = 0 does nothing.
 * Errors: those of hull_compute_host; EINVAL for count < 0 or NULL arrays. */
hull_status hull_compute_host_multi(hull_ctx *ctx, int32_t count, const int32_t *const *h_xy,
                                    const int64_t *n, int32_t *const *h_out, const int64_t *cap,
                                    int64_t *h_count, void *stream);

/* B independent hulls in one call (Section 2.1's pipeline on every
 * instance).  Instances of at least hull_config.batched_seg_min points (or
 * the autotuned / default boundary) take the segmented path: two flat
 * streaming passes over all their 16,384-point tiles at once (extremes;
 * witness test and filter polygon), with one block per instance for its
 * plan and, after the passes, for its sort, second round and chains.  The
 * others go one block per instance through a persistent launch per size
 * bucket (up to 16,384 points, more), instances taken largest first, on
 * the context's second stream.  d_offsets: device int64[B+1], instance b is points
 * [d_offsets[b], d_offsets[b+1]) of d_xy (non-decreasing, d_offsets[0] = 0).
 * Vertex indices are relative to their instance and are written to d_out at
 * d_out_offsets[b] (device int64[B+1], written by the call;
 * d_out_offsets[B] = total vertices).  cap bounds the total (HULL_ECAPACITY
 * leaves d_out untouched but still writes d_out_offsets).  Total points must
 * be < 2^30 and every instance at most hull_batched_max_instance() points
 * (else HULL_EINVAL).  Copies d_offsets to the host and synchronises
 * `stream`. */
hull_status hull_compute_batched(hull_ctx *ctx, const int32_t *d_xy, const int64_t *d_offsets,
                                 int32_t B, int32_t *d_out, int64_t cap, int64_t *d_out_offsets,
                                 void *stream);

/* ---- learned filter proposal (the project's addition beside Section 3.1's
 * quadrilateral): an MLP 64 -> 128 -> 128 -> 32 (ReLU) scores 32 directions
 * from features of a strided sample of the input; the filter polygon is the
 * exact hull of the quadrilateral's corners and the extremes of the 8 best
 * directions (used when it encloses more area than the quadrilateral).
 * Enabled by hull_config.proposal = 1 once parameters are set or loaded;
 * without parameters the quadrilateral is used.  Parameters (FP32 master,
 * FP16 at inference) are laid out W1[128][64], b1[128], W2[128][128],
 * b2[128], W3[32][128], b3[32]. ---- */
int64_t hull_mlp_num_params(void);
hull_status hull_mlp_set_params(hull_ctx *ctx, const float *h_params, int64_t count);
hull_status hull_mlp_get_params(const hull_ctx *ctx, float *h_params, int64_t count);
/* Checkpoint: 8 uint32 header (magic "GBHL", version 1, 64, 128, 128, 32,
 * parameter count, CRC-32 of the parameters) then the FP32 parameters. */
hull_status hull_save_proposal(const hull_ctx *ctx, const char *path);
hull_status hull_load_proposal(hull_ctx *ctx, const char *path);
/* Features of the strided sample i_k = floor(k n / S), S = min(n, 16384)
 * (d_feat device float[64]: 32 angular bins
 * of point fractions, then 32 of maximum radius over the largest) and the
 * sample's extreme point per direction j (d_ext int32[32] indices,
 * d_ext_xy int32[32][2]); u_j = (cos 2 pi j/32, sin 2 pi j/32). */
hull_status hull_learned_features(hull_ctx *ctx, const int32_t *d_xy, int64_t n, float *d_feat,
                                  int32_t *d_ext, int32_t *d_ext_xy, void *stream);
/* Training labels: h_labels[j] = fraction of points strictly inside
 * hull(quadrilateral corners + extreme j) minus the fraction strictly inside
 * the quadrilateral (*h_quad_frac), counted exactly. */
hull_status hull_learned_labels(hull_ctx *ctx, const int32_t *d_xy, int64_t n, float *h_labels,
                                float *h_quad_frac, void *stream);
/* Forward pass of B feature rows (d_X device float[B][64]) into d_Z
 * (device float[B][32]); gradient of the mean squared error against d_Y
 * (device float[B][32]) into h_grad (host, hull_mlp_num_params floats);
 * one Adam step (beta 0.9 / 0.999, eps 1e-8) at learning rate lr. */
hull_status hull_mlp_forward(hull_ctx *ctx, const float *d_X, int32_t B, float *d_Z, void *stream);
hull_status hull_mlp_gradient(hull_ctx *ctx, const float *d_X, const float *d_Y, int32_t B,
                              float *h_grad, float *h_loss, void *stream);
hull_status hull_mlp_train_step(hull_ctx *ctx, const float *d_X, const float *d_Y, int32_t B,
                                float lr, float *h_loss, void *stream);

/* Largest instance size hull_compute_batched accepts. */
int64_t hull_batched_max_instance(void);

/* Survivor counts and extremes of the last hull_compute (collect_stats=1). */
hull_status hull_last_stats(const hull_ctx *ctx, hull_stats *out);

/* Per-stage device time of hull_compute calls, measured with CUDA events
 * recorded on the call's stream between the pipeline's kernels (profiling
 * must be enabled with hull_set_profiling; accumulation restarts then). */
#define HULL_NUM_STAGES 12
typedef struct {
  int64_t calls;                 /* hull_compute calls accumulated */
  int64_t radix_calls;           /* of those, calls sorted by the radix passes (the rerun of a
                                    call whose bins the bucket sort could not take) */
  int64_t sort_passes;           /* radix passes that did work, summed over calls */
  int64_t points;                /* input points, summed */
  int64_t survivors;             /* first-round survivors, summed (counted only by a context
                                    with collect_stats; 0 otherwise) */
  int64_t second_round;          /* second-round survivors, summed */
  double ms[HULL_NUM_STAGES];    /* per stage; with the bucket sort (the default): polygon
                                    (single-read front: the sample polygon; empty on the
                                    two-read front), extremes (single-read front: the extremes
                                    pass that filters with the polygon), witnesses (the
                                    sample's best witness per bin), filter (the
                                    fused filter: witness test, filter polygon, compaction, bin
                                    scan), scatter (survivors into coarse bins), split (coarse bins
                                    into bins, their aggregates, the groups' prefixes), sort (groups
                                    sorted, second round), 3 empty slots, regions (compaction),
                                    final; on the radix passes: extremes, filter, radix pass 0..7,
                                    regions, final */
  int64_t witness_survivors;     /* survivors of the fused filter (the bucket sort's input),
                                    summed; the first-round survivors on the radix passes */
  int64_t raw_survivors;         /* single-read front: points on or outside the sample polygon
                                    (the fused filter's input), summed; 0 for calls on the
                                    two-read front */
  int64_t single_read_calls;     /* calls that took the single-read front */
} hull_profile;

hull_status hull_set_profiling(hull_ctx *ctx, int enable);
hull_status hull_get_profile(const hull_ctx *ctx, hull_profile *out);

/* ---- allocation-free entry point (no counterpart in the paper) ----
 * For callers that must not allocate device memory: code that runs where
 * cudaMalloc is forbidden or unsafe (a host callback, a memory-pool hook, a
 * plug-in whose host application owns the device memory budget) or that
 * cannot afford the device-wide synchronisation cudaMalloc/cudaFree may
 * imply.  Same computation and result as hull_compute, but it needs no
 * context and allocates nothing (no cudaMalloc, cudaFree, pinned buffer or
 * allocating library call): its scratch memory is one file-scope device
 * array of HULL_NOALLOC_SCRATCH_BYTES that every GPU which loads this
 * library holds until the process exits.
 *   - n must be <= HULL_NOALLOC_MAX_POINTS, else HULL_EINVAL;
 *   - runs on the current CUDA device; d_xy, d_out and h_count as in
 *     hull_compute; synchronises `stream` before returning;
 *   - all calls on a device share the array, which keeps the last call's
 *     contents; each call clears what must start at zero before using it;
 *     calls whose GPU work overlaps (other streams, other host threads on
 *     the same device) race on the array and must be serialised;
 *   - the first call on each device does a one-time set-up with that device
 *     current (it resolves the array's device address and sets kernel
 *     attributes); make that first call before any stream capture. */
#define HULL_NOALLOC_MAX_POINTS 65536
#define HULL_NOALLOC_SCRATCH_BYTES (6u << 20)
hull_status hull_compute_noalloc(const int32_t *d_xy, int64_t n, int32_t *d_out, int64_t cap,
                                 int64_t *h_count, void *stream);

/* Short English text for a status code (static storage). */
const char *hull_status_string(hull_status s);

/* ---- stage entry points: each runs one step of the pipeline on its own,
 * so that every step can be checked against a CPU restatement. ---- */

/* Section 2.1 step 1 / Section 3.1: h_ext[4] (host) = indices of P_minx =
 * argmin (x, y), P_maxx = argmax (x, y), P_miny = argmin (y, x), P_maxy =
 * argmax (y, x), ties to the smallest index; n >= 1.  ERANGE is reported
 * after h_ext is written. */
hull_status hull_stage_extremes(hull_ctx *ctx, const int32_t *d_xy, int64_t n, int32_t *h_ext,
                                void *stream);

/* Section 2.1 step 2 / Section 3.1: indices of the points not strictly
 * inside the quadrilateral P_minx, P_miny, P_maxx, P_maxy (nothing is
 * discarded when it has fewer than three distinct corners), ascending, into
 * d_keep (device int32[n]); *h_s = their count. */
hull_status hull_stage_filter(hull_ctx *ctx, const int32_t *d_xy, int64_t n, int32_t *d_keep,
                              int64_t *h_s, void *stream);

/* Section 2.1 step 4 / Section 3.3: stable ascending sort of m (key, value)
 * pairs: d_keys (device uint64[m]) and d_vals (device uint32[m]) are sorted
 * in place (the workspace holds the ping-pong copies).  m < 2^30. */
hull_status hull_stage_sort(hull_ctx *ctx, uint64_t *d_keys, uint32_t *d_vals, int64_t m,
                            void *stream);

/* Section 2.1 step 4 / Section 3.3 as the hull pipeline runs it: the
 * bucket sort of m (key, value) pairs, ascending by key and, among equal
 * keys, by value -- the stable sort of hull_stage_sort whenever the values
 * increase in input order, as the first round's survivor indices do.
 * Pairs are binned by the top bits of the key and each group of bins is
 * sorted in shared memory; if some bin cannot be (too many equal or nearly
 * equal keys) the pairs are sorted by hull_stage_sort instead and
 * *h_fallback (host, may be NULL) is set to 1, else 0.  d_keys (device
 * uint64[m]) and d_vals (device uint32[m]) are sorted in place.
 * m < 2^30. */
hull_status hull_stage_bucket_sort(hull_ctx *ctx, uint64_t *d_keys, uint32_t *d_vals, int64_t m,
                                   int32_t *h_fallback, void *stream);

/* The largest number of pairs the bucket sort orders in one block's shared
 * memory: a bin above it is split once more by its next key bits, and a
 * piece of it still above it sends the call to the radix passes. */
int64_t hull_bucket_group_cap(void);

/* Section 2.1 steps 5-7 / Figure 2: the second-round filter over m points
 * already sorted by (x, y, index): d_xy (device int32[m][2]) in that order
 * and d_idx (device int32[m]) their labels.  Writes the kept labels of the
 * lower region (right of P_0 -> P_l) to d_lower and of the upper region to
 * d_upper (device int32[m] each), in list order; counts in *h_lower,
 * *h_upper. */
hull_status hull_stage_second_round(hull_ctx *ctx, const int32_t *d_xy, const int32_t *d_idx,
                                    int64_t m, int32_t *d_lower, int64_t *h_lower,
                                    int32_t *d_upper, int64_t *h_upper, void *stream);

/* Section 2.1 steps 1-4 on n >= 1 points (d_xy device int32[n][2]): the
 * extremes, the quadrilateral filter and the sort, through the stable
 * compaction and the radix passes.  Writes the first-round survivors in
 * (x, y, index) order as points to d_xy_out (device int32[cap][2]) and
 * their input indices to d_idx_out (device int32[cap]); *h_count receives
 * their number.  HULL_ECAPACITY when cap is smaller (count still set). */
hull_status hull_stage_sorted_survivors(hull_ctx *ctx, const int32_t *d_xy, int64_t n, int32_t *d_xy_out,
                                        int32_t *d_idx_out, int64_t cap, int64_t *h_count, void *stream);

/* Section 3.4's chunked second round, the paper's own parallelisation of
 * Figure 2, as an ablation of the exact scan: over m >= 1 points sorted by
 * (x, y, index) (d_xy device int32[m][2], d_idx device int32[m] their
 * labels), each region's points are split into block_size (1 .. 1024) runs
 * of ceil(m_region / block_size) consecutive points and Figure 2 runs over
 * every run on its own from P_temp = P_0 (one thread per run, one block per
 * region, as the paper does).  block_size = 1 is the exact second round.
 * Writes the kept labels of the lower / upper region to d_lower / d_upper
 * (device int32[m] each) in list order; counts in *h_lower, *h_upper. */
hull_status hull_stage_second_round_chunked(hull_ctx *ctx, const int32_t *d_xy, const int32_t *d_idx,
                                            int64_t m, int32_t block_size, int32_t *d_lower,
                                            int64_t *h_lower, int32_t *d_upper, int64_t *h_upper,
                                            void *stream);

/* The front of hull_compute on n points (d_xy device int32[n][2]):
 * extremes, quadrilateral filter, sort and the second-round filter
 * (Section 2.1 steps 1-7, Figure 2), fused as in hull_compute.  Writes the
 * labels (input indices) of the points the second round keeps in the lower
 * region to d_lower (device int32[lower_cap]) and in the upper region to
 * d_upper (device int32[upper_cap]), each in sorted (x, y, index) order
 * without P_0 and P_l; h_counts (host int64[2]) receives both counts and
 * *h_fallback (if not NULL) whether the call was rerun on the radix passes.
 * HULL_ECAPACITY when a list does not fit (counts still set, buffers
 * untouched).  Synchronises `stream`. */
hull_status hull_stage_regions(hull_ctx *ctx, const int32_t *d_xy, int64_t n, int32_t *d_lower,
                               int64_t lower_cap, int32_t *d_upper, int64_t upper_cap,
                               int64_t *h_counts, int32_t *h_fallback, void *stream);

/* Section 2.1 step 8: stack-based chains over m >= 2 distinct points in
 * lexicographic order (d_xy device int32[m][2]).  d_out (device int32[cap])
 * receives the lower chain's positions (first to last point, left turns)
 * followed by the upper chain's positions reversed without its endpoints;
 * *h_lower and *h_upper receive both chain lengths (endpoints included). */
hull_status hull_stage_chain(hull_ctx *ctx, const int32_t *d_xy, int64_t m, int32_t *d_out,
                             int64_t cap, int64_t *h_lower, int64_t *h_upper, void *stream);

/* Section 2.1 steps 1-7 with the paper's own ordering (Sections 3.2-3.3:
 * the first-round survivors sorted by angle; Figure 2 as printed: P_l the
 * point farthest from P_0, the right region walked forward from P_0, the
 * left region backward from the last point), on n >= 1 points (d_xy device
 * int32[n][2], 8-byte aligned).  The anchor P_0 is P_miny = argmin (y, x,
 * index); points equal to it are left out; the order is exact (an integer
 * angle key, never a rounded angle) with equal angles nearer first, then by
 * index.  Writes [P_0, the points by angle] as input indices to d_order
 * (device int32[cap]) and 1 / 0 to d_keep (device uint8[cap]) for each
 * position the second round keeps / discards (P_0, P_l and the last point
 * are always kept); *h_m receives the number of positions and *h_l the
 * position of P_l (-1 when P_0 is the only distinct point).  HULL_ECAPACITY
 * when cap < *h_m (nothing written); HULL_ERANGE for coordinates beyond
 * +-2^29; HULL_ENOMEM when its scratch cannot be allocated.  Its scratch
 * (a few tens of bytes per point) lives in a context-owned area that the first
 * call of a given size allocates and later calls reuse (it grows, after a
 * device synchronisation, only when a larger call comes); synchronises
 * `stream`. */
hull_status hull_stage_angular(hull_ctx *ctx, const int32_t *d_xy, int64_t n, int32_t *d_order,
                               uint8_t *d_keep, int64_t cap, int64_t *h_m, int64_t *h_l, void *stream);

/* The convex hull by the paper's angular variant, steps 1-8: the front of
 * hull_stage_angular, then step 8 (the hull of the points the second round
 * keeps) on the device, over those points in angular order, with the same
 * chains as hull_compute.  d_xy: device int32[n][2] (8-byte aligned),
 * n >= 0.  d_out: device int32[cap] receiving the hull's vertex indices,
 * counter-clockwise from the lexicographic minimum, strict vertices only;
 * among equal points the first in angular order among those the second
 * round keeps is reported (the one Graham's scan keeps; the backward walk
 * keeps the largest index of equal points).  *h_count receives the hull size on HULL_OK and on
 * HULL_ECAPACITY (then d_out is untouched).  Scratch as hull_stage_angular,
 * plus about 40 bytes per point, in the same context-owned area; synchronises
 * `stream`. */
hull_status hull_compute_angular(hull_ctx *ctx, const int32_t *d_xy, int64_t n, int32_t *d_out, int64_t cap,
                                 int64_t *h_count, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* GBHULL_H */
