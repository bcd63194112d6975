/*
 * convhull.h -- C ABI of the GB300 octagon-filter convex-hull library.
 *
 * Method: Carrasco, Ferrada, Navarro, Hitschfeld, "An Evaluation of GPU
 * Filters for Accelerating the 2D Convex Hull" (arXiv 2303.10581),
 * Algorithm 1: findingPolygon -> buildingFilter ->
 * compactingFilteredPoints -> convexHull_algorithm.  Every step runs in
 * hand-written sm_103a CUDA kernels; nothing here falls back to the host.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Points are packed binary32 pairs (x, y), x at the lower address:
 *    `pts` holds 2*n floats.  Coordinates must be finite.  8-byte alignment
 *    is required, 16-byte alignment is preferred (vector loads).
 *  - Every array argument is a DEVICE pointer owned by the caller; the
 *    library allocates nothing.  `ws` is caller-owned device scratch of at
 *    least ch_workspace_size() bytes, 256-byte aligned; it must be zeroed
 *    once (ch_workspace_init) before its first use and then belongs to the
 *    library until the calls that use it have completed.  One workspace
 *    serves one stream at a time.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Calls are asynchronous on that stream: outputs, including
 *    counts, are written to device memory and are valid once the stream
 *    reaches the call.
 *  - Argument errors are detected on the host and returned at once; no work
 *    is enqueued then.  Errors found on the device (non-finite input, a
 *    look-back wait that timed out) are recorded in `ws` and reported by
 *    ch_last_error(); outputs of a failed call are unspecified.
 *  - Host threads: apart from thread-safe caches of device properties, the
 *    compute entry points keep no host state between calls, so several
 *    host threads may drive them at once, each on its own stream and
 *    workspace.  Three settings are process-wide instead:
 *    the compaction schedule (ch_filter_variant), the batched launch grids
 *    (ch_tune_set) and the instrumentation (ch_probe_start/stop).  The two
 *    settings are atomics read when a call enqueues its kernels, so a call
 *    running concurrently with a change uses either the old or the new
 *    value (results are the same either way, only the schedule differs);
 *    set them before the calls they are meant for.  The probe's event
 *    lists are meant for one host thread at a time: while a probe is
 *    active, make the calls it should time from the thread that started
 *    it, and no calls from others.
 *  - Point indices are uint32: n < 2^32 (ch_hull: n < 2^30).
 *  - Orientation signs are exact (binary32 fast test with a proven error
 *    bound, then binary64, then error-free expansion arithmetic).
 */
#ifndef CONVHULL_H
#define CONVHULL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    CH_OK = 0,
    CH_ERR_ARG = 1,         /* bad pointer, size or alignment               */
    CH_ERR_NONFINITE = 2,   /* a coordinate is NaN or infinite              */
    CH_ERR_CAPACITY = 3,    /* workspace too small / n beyond the limit     */
    CH_ERR_CUDA = 4,        /* a CUDA runtime call failed                   */
    CH_ERR_TIMEOUT = 5,     /* a bounded device-side wait gave up           */
    CH_ERR_UNSUPPORTED = 6  /* device is not sm_103 or feature unavailable  */
} ch_status;

/* Bytes of workspace needed for point sets of up to n points in total,
 * split into up to num_sets sets (num_sets = 1 for the single-set calls).
 * No CUDA work.  Returns CH_ERR_ARG for negative sizes or a NULL `bytes`. */
ch_status ch_workspace_size(int64_t n, int64_t num_sets, size_t *bytes);

/* Zero a workspace of ws_bytes bytes on `stream` (one cudaMemsetAsync).
 * Needed once before first use, and again after a call reported an error. */
ch_status ch_workspace_init(void *ws, size_t ws_bytes, void *stream);

/* Sec. 3.1 (findingPolygon): the eight polygon vertices.
 * ext8[0..7] receives point indices in counter-clockwise order
 *   R = argmax x, TR = argmax fl(x+y), T = argmax y, TL = argmin fl(x-y),
 *   L = argmin x, BL = argmin fl(x+y), B = argmin y, BR = argmax fl(x-y),
 * the corner points being the points closest in Manhattan distance to the
 * bounding-box corners.  fl() is binary32 round-to-nearest.  Ties go to the
 * lowest index; -0 and +0 compare equal.  n >= 1.  A NaN or infinite
 * coordinate sets CH_ERR_NONFINITE in ws (ext8 is then unspecified). */
ch_status ch_extremes(const float *pts, int64_t n, uint32_t *ext8,
                      void *ws, size_t ws_bytes, void *stream);

/* Sec. 3.2 (buildingFilter + compactingFilteredPoints): discard the points
 * lying strictly inside the closed polygon pts[ext8[0]], ..., pts[ext8[7]]
 * (strictly left of every edge of non-zero length), keep all others, and
 * compact the kept ones stably.  surv_idx (capacity n) receives the kept
 * indices in ascending order, surv_pts (capacity 2n floats, may be NULL)
 * their coordinates, and *surv_count (device) their number.  ext8 is a
 * device array, normally the output of ch_extremes, but any eight indices
 * < n are accepted, in any order (repeated, interior or clockwise vertices
 * included): the result is exact for the vertex sequence given.  An index
 * >= n sets CH_ERR_ARG in ws and writes a zero count.  n == 0 writes a
 * zero count. */
ch_status ch_filter(const float *pts, int64_t n, const uint32_t *ext8,
                    uint32_t *surv_idx, float *surv_pts, uint32_t *surv_count,
                    void *ws, size_t ws_bytes, void *stream);

/* Sec. 3.1 + Sec. 3.2 in one call (Algorithm 1, steps 1-3): ext8 (device,
 * 8 entries) receives the eight vertices exactly as ch_extremes gives
 * them, and surv_idx / surv_pts / *surv_count the survivors of the filter
 * with that polygon exactly as ch_filter gives them.  On sets of at least
 * 2^22 points with the two-pass schedule (ch_filter_variant 0) it runs the
 * speculative single sweep: a first kernel builds an octagon P0 from a
 * 65,536-point sample; the extremes sweep also writes, as candidates, the
 * points it cannot prove strictly inside P0; when its last block proves
 * P0 inside the final octagon (exact signs) and no candidate segment
 * overflowed, only the candidates are tested and written, so the points
 * are read once.  Otherwise the filter's two passes run over all points.
 * The results are the same either way.  Errors as ch_extremes and
 * ch_filter; n == 0 writes a zero count. */
ch_status ch_extremes_filter(const float *pts, int64_t n, uint32_t *ext8, uint32_t *surv_idx,
                             float *surv_pts, uint32_t *surv_count, void *ws, size_t ws_bytes,
                             void *stream);

/* Algorithm 1 end to end on the device: extremes, filter, then Andrew's
 * monotone chain over the survivors (Sec. 3.3; the paper hands this step to
 * a CPU library, here it stays on the GPU).  hull_idx (capacity n)
 * receives original point indices counter-clockwise, starting at the
 * lexicographically smallest (x, y) vertex; equal points count once (the
 * lowest index is reported); points on a hull edge are not vertices.
 * *hull_count (device) receives the vertex count: 0 for n == 0, 1 when all
 * points coincide, 2 when all are collinear.  Before the sort the hull step
 * throws survivors away again (not in the paper; the hull is the same): a
 * fan of triangles around the bounding-box centre whose vertices are the
 * farthest sampled survivors of angular bins, and, when that leaves at least
 * 2^19 points (CH_TUNE_FAN2_MIN_LOG2), a second fan over those with eight
 * times as many bins; a survivor strictly inside a triangle (exact signs) is
 * no hull vertex. */
ch_status ch_hull(const float *pts, int64_t n, uint32_t *hull_idx, uint32_t *hull_count,
                  void *ws, size_t ws_bytes, void *stream);

/* Many independent sets in one call.  Set b is pts[offsets[b] .. offsets[b+1])
 * (offsets is a DEVICE array of num_sets+1 non-decreasing int64, offsets[0]
 * = 0).  Set b's hull is written, as set-local indices in the same order as
 * ch_hull, to hull_idx[hull_offsets[b] ..], with hull_offsets (device,
 * num_sets+1 entries) the exclusive prefix sum of the hull sizes.
 * hull_idx capacity: offsets[num_sets] entries.  ws must be sized with
 * ch_workspace_size(N, num_sets) for some N >= offsets[num_sets]; since the
 * offsets live on the device, the host derives the point capacity from
 * ws_bytes and the device checks the offsets against it.  num_sets == 0
 * writes hull_offsets[0] = 0.  Device-side errors (reported by
 * ch_last_error; hull_offsets are then all 0): malformed offsets
 * (offsets[0] != 0, a negative or decreasing entry) CH_ERR_ARG, more points
 * than the workspace holds CH_ERR_CAPACITY.  A set with a non-finite
 * coordinate gets an empty hull and CH_ERR_NONFINITE is reported; the
 * other sets are still computed.  Total points < 2^30.  Not part of the
 * paper: the batched form of the same path (Algorithm 1 per set). */
ch_status ch_hull_batched(const float *pts, const int64_t *offsets, int32_t num_sets,
                          uint32_t *hull_idx, int64_t *hull_offsets,
                          void *ws, size_t ws_bytes, void *stream);

/* The filter polygon generalised to K directions (the polygon a learned
 * proposal picks; Sec. 3.1-3.2 with K in place of 8).  dirs is a DEVICE
 * array of K (c_k, s_k) binary32 pairs, counter-clockwise, |c_k|, |s_k| <= 1;
 * K is 8, 16, 32 or 64 (CH_ERR_ARG otherwise).  Vertex k is the point with
 * the largest key fl(fl(c_k x) + fl(s_k y)) (binary32, lowest index on
 * ties); with the eight directions (1,0), (1,1), (0,1), (-1,1), (-1,0),
 * (-1,-1), (0,-1), (1,-1) these are the octagon's keys and vertices.  A
 * point is discarded when it is strictly left of every edge of non-zero
 * length of the closed vertex sequence (exact sign); the kept points are
 * compacted as by ch_filter (surv_idx ascending, surv_pts may be NULL,
 * *surv_count on the device).  ext_out (device, K entries, may be NULL)
 * receives the vertex indices.  Non-finite input: CH_ERR_NONFINITE in ws,
 * zero count.  Not part of the paper's method: its generalisation. */
ch_status ch_filter_kgon(const float *pts, int64_t n, const float *dirs, int32_t K, uint32_t *ext_out,
                         uint32_t *surv_idx, float *surv_pts, uint32_t *surv_count,
                         void *ws, size_t ws_bytes, void *stream);

/* ch_hull with the K-direction polygon of ch_filter_kgon as its filter
 * (same hull: every polygon vertex is an input point).  The hull step
 * sorts and chains every survivor (no fan test). */
ch_status ch_hull_kgon(const float *pts, int64_t n, const float *dirs, int32_t K, uint32_t *hull_idx,
                       uint32_t *hull_count, void *ws, size_t ws_bytes, void *stream);

/* ch_hull with a second filter polygon between the octagon and the hull
 * step (the paper's Sec. 3.1 idea with K directions, applied to what the
 * octagon leaves): after the octagon's count pass, vertex k of the K-gon
 * is the survivor with the largest key fl(fl(c_k x) + fl(s_k y)) (dirs as
 * in ch_filter_kgon; lowest index on ties), and survivors strictly left of
 * every edge of non-zero length of that vertex sequence are dropped too;
 * then the fan test, sort and chain of ch_hull.  K in {8, 16, 32, 64};
 * K = 8 adds no polygon (ch_hull exactly; dirs may be NULL).  The hull is
 * ch_hull's.  ext_out (device, K entries, may be NULL) receives the K-gon's
 * vertex indices when the second polygon ran: not when the speculative
 * sweep served the filter (ch_hull_counts) or the single-pass schedule is
 * set, which leave no keep bits to refine.  Errors as ch_hull and
 * ch_filter_kgon. */
ch_status ch_hull_octagon_kgon(const float *pts, int64_t n, const float *dirs, int32_t K, uint32_t *ext_out,
                               uint32_t *hull_idx, uint32_t *hull_count, void *ws, size_t ws_bytes,
                               void *stream);

/* The learned proposal end to end without a host synchronisation (not in
 * the paper): one block computes the features (as ch_kgon_features) and
 * the MLP (as ch_mlp_forward, each output's sum spread over a warp, so its
 * rounding may differ in the last bits), then K from the arg-max of the four K-logits
 * and the directions at angles 2 pi k / K + offset_k pi / K (offsets
 * clipped to +-0.45; cos and sin in binary64, rounded once; a multiple of
 * pi / 4 with zero offset takes the octagon's integer direction), then
 * ch_hull_octagon_kgon with that polygon (K = 8: ch_hull).  params: device,
 * the MLP's BF16 parameters (ch_mlp_forward).  dirs_out (device, 128
 * floats, may be NULL: the K directions as (cos, sin) pairs, zeros after
 * them) and k_out (device, may be NULL) receive the choice.
 * The hull is ch_hull's whatever the MLP outputs. */
ch_status ch_hull_learned(const float *pts, int64_t n, const void *params, float *dirs_out, int32_t *k_out,
                          uint32_t *hull_idx, uint32_t *hull_count, void *ws, size_t ws_bytes, void *stream);

/* ---- launch tuning of ch_hull_batched ---------------------------------
 * Launch shapes of the batched kernels; results do not depend on them
 * (every such kernel walks tiles grid-stride, by ticket or over its own
 * range, and the fan's vertices are input points whatever the sample).
 * 0 restores the built-in choice.  Process-wide (see "Host threads"
 * above), host-only; CH_ERR_ARG for an unknown knob or a value outside the
 * knob's range.  The Python package's autotuner sweeps these on a
 * workload and caches the best in JSON. */
typedef enum {
    CH_TUNE_BX_EXTREMES = 0,    /* extremes sweep, blocks per SM 1..64 (default 8)          */
    CH_TUNE_BX_FILTER = 1,      /* filter count and scatter, blocks per SM (default: occupancy) */
    CH_TUNE_BX_SORT_PASS = 2,   /* radix-sort passes, blocks per SM (default: occupancy)     */
    CH_TUNE_BX_EMIT = 3,        /* chain compaction, blocks per SM (default 4)              */
    CH_TUNE_BX_FAN_STRIDE = 4,  /* the fan's bins sample every k-th tile of a set, 1..64 (default 2) */
    CH_TUNE_BX_FAN_CHUNK = 5,   /* tiles per work item of the fan refine: 8, 16, 32 or 64 (default 64) */
    CH_TUNE_BX_EXT_ITEMS = 6,   /* points per thread per 4096-point tile of the extremes sweep:
                                   4, 8 or 16, i.e. blocks of 1024, 512 or 256 threads (default 16) */
    CH_TUNE_FAN2_MIN_LOG2 = 7,  /* single-set hull step: the fan's second level runs when the first
                                   leaves at least 2^value points, 10..31 (default 19); sets of
                                   fewer than 2^19 points have no second level */
    CH_TUNE_COUNT = 8
} ch_tune_knob;
ch_status ch_tune_set(int32_t knob, int32_t value);
ch_status ch_tune_get(int32_t knob, int32_t *value);

/* ---- learned proposal of the K-direction polygon (not in the paper: its
 * extension to more directions, picked per point set) ---------------------
 * Features of a point set: a 32 x 32 occupancy grid of a sample of
 * m = min(n, 4096) points (indices floor(j n / m)) over the sample's
 * bounding box, cell = min(31, floor(fl(fl(x - xmin) * fl(32 / w)))) per
 * axis (w the box width, 0 scale when w = 0), as fractions of m.  feat:
 * DEVICE, 1024 floats (row = y cell).  One block; CH_ERR_ARG for n < 1. */
ch_status ch_kgon_features(const float *pts, int64_t n, float *feat, void *stream);

/* The MLP 1024 -> 64 -> 64 -> 68 (4 logits of K in {8, 16, 32, 64}, 64
 * angular offsets), ReLU between, BF16 weights, FP32 accumulation.
 * params: DEVICE bf16[ch_mlp_param_count()], row-major
 * W1[64][1024] b1[64] W2[64][64] b2[64] W3[68][64] b3[68].  X: DEVICE
 * float[B][1024]; H1, H2: float[B][64]; OUT: float[B][68] (DEVICE). */
int32_t ch_mlp_param_count(void);
ch_status ch_mlp_forward(const float *X, int32_t B, const void *params, float *H1, float *H2, float *OUT,
                         void *stream);

/* One Adam step (beta 0.9, 0.999, eps 1e-8, bias-corrected with `step`
 * >= 1) on the batch: loss = mean over the batch of the softmax
 * cross-entropy of OUT[0:4] against label[b] (0..3) plus
 * lam * mask[b] * mean_j (OUT[4+j] - off[b][j])^2.  master, adam_m, adam_v:
 * DEVICE float[param count] (FP32 master weights and moments); params
 * receives the BF16 copy of the updated master weights.  scratch: DEVICE
 * float[ch_mlp_scratch_floats(B)]; loss: DEVICE float[B] (per sample). */
ch_status ch_mlp_train_step(const float *X, int32_t B, const int32_t *label, const float *off, const float *mask,
                            float lam, void *params, float *master, float *adam_m, float *adam_v, int32_t step,
                            float lr, float *scratch, float *loss, void *stream);
int64_t ch_mlp_scratch_floats(int32_t B);

/* Waits for `stream`, then returns and clears the first device-side error
 * recorded in ws since the last call (CH_OK if none). */
ch_status ch_last_error(void *ws, void *stream);

/* ch_filter for callers that cannot allocate device memory and cannot pass
 * a workspace -- e.g. code inside a host framework that owns every device
 * allocation, or a path under a fixed memory budget or a latency budget
 * that cudaMalloc's implicit synchronisation would break.  The paper has no
 * counterpart; this is a packaging of the same filter.
 * Same arguments, results and host-side error codes as ch_filter, without
 * ws: the scratch lives in a 160 KiB static device array inside the
 * library, held by every GPU that loads it until the process exits.  n is
 * limited to 2^26 = 67,108,864 points (CH_ERR_CAPACITY beyond).  Allocates
 * nothing.  The first call on each device looks up the array's device
 * address (with that device current) and keeps it; make that first call
 * before any stream capture.  cudaDeviceReset invalidates the kept address:
 * do not call this entry point after a reset.  All calls share the array:
 * calls whose work overlaps on the GPU race and must be serialised by the
 * caller.  Device-side errors (an ext8 index >= n: CH_ERR_ARG; a look-back
 * wait that gave up: CH_ERR_TIMEOUT) are reported in the count, which then
 * reads 0x80000000 | code (a valid count is below 2^26); surv_idx and
 * surv_pts are then unspecified. */
ch_status ch_filter_noalloc(const float *pts, int64_t n, const uint32_t *ext8,
                            uint32_t *surv_idx, float *surv_pts, uint32_t *surv_count,
                            void *stream);

/* Compaction strategy of the filter (Sec. 3.2) for later ch_filter and
 * ch_hull calls of this process; results are identical, only the schedule
 * differs.  0 (default): two passes -- a streaming count of the survivors
 * of every 4096-point tile, a scan of the counts, and a scatter pass that
 * revisits only tiles with survivors.  1: one pass -- tiles in ticket order
 * with a decoupled look-back for their output offsets.  CH_ERR_ARG for any
 * other value.  Host-only; process-wide (see "Host threads" above). */
ch_status ch_filter_variant(int32_t variant);

/* ---- instrumentation (not part of the paper's method) ------------------
 * Kernel identifiers of the path. */
typedef enum {
    CH_K_EXTREMES = 0,   /* Sec. 3.1 sweep (+ polygon build in its last block) */
    CH_K_OCTAGON = 1,    /* polygon build for ch_filter                        */
    CH_K_FILTER = 2,     /* Sec. 3.2 fused test + stable compaction            */
    CH_K_SORT_HIST = 3,  /* digit histograms of the survivor keys              */
    CH_K_SORT_PASS = 4,  /* one radix-sort pass                                 */
    CH_K_CHAIN = 5,      /* Sec. 3.3 chunk chains + tree merges                 */
    CH_K_EMIT = 6,       /* compaction of the chain ranges                      */
    CH_K_FINISH = 7,     /* hull assembly                                       */
    CH_K_KGON = 8,       /* hull step: fan test of the octagon survivors
                            (runs between FILTER's count and scatter passes;
                            its second level after the scatter) */
    CH_K_COUNT = 9
} ch_kernel_id;

/* Start timing: every later launch group of a kernel id whose bit (1 << id)
 * is set in kernel_mask is bracketed by two CUDA events recorded on its
 * launch stream, for at most max_launches groups per id.  A group is the
 * kernels one step launches back to back under that id: one for
 * EXTREMES, OCTAGON, SORT_HIST, SORT_PASS (one per pass), FINISH; two for
 * EMIT (offsets, copy); two for FILTER with the two-pass schedule (count,
 * scatter; in ch_hull each is its own group, KGON runs between them), one
 * with the single pass; two for CHAIN (chains, tree merge); for KGON three
 * (fan vertices, estimate, refine of the keep decisions; the count pass
 * gathers the bins) and four for its second level (sub-bin maxima,
 * vertices, test, compaction).  Kernel-launch
 * counting for all ids restarts at zero.  Host-only bookkeeping; creates
 * the events.  Process-wide: one probe at a time, driven from one host
 * thread (see "Host threads" above). */
ch_status ch_probe_start(uint32_t kernel_mask, int32_t max_launches);

/* After a ch_hull call for n points on ws has completed (waits for
 * `stream`): counts[0] = points that survived the octagon filter,
 * counts[1] = points the hull step sorted (fewer when its fan of triangles
 * around the bounding-box centre removed some), counts[2] = 1 when the
 * speculative single sweep served the filter (the extremes sweep proved
 * every point but its candidates strictly inside the octagon, so the
 * filter read only the candidates), else 0, counts[3] = points left by the
 * fan's first level (the input of its second level over the survivors,
 * with kFan2Sub times as many bins, when that ran; else counts[1]).
 * counts holds 4 entries.  Instrumentation; CH_ERR_ARG / CH_ERR_CAPACITY
 * as for ch_hull. */
ch_status ch_hull_counts(void *ws, size_t ws_bytes, int64_t n, uint32_t *counts, void *stream);

/* Stop timing: waits for the recorded events, writes per kernel id the summed
 * event-measured milliseconds (ms[CH_K_COUNT], 0 when not timed) and the
 * number of kernels launched under it since ch_probe_start, in every
 * stream (launches[CH_K_COUNT]), and releases the events.  Either pointer
 * may be NULL. */
ch_status ch_probe_stop(double *ms, int64_t *launches);

#ifdef __cplusplus
}
#endif

#endif /* CONVHULL_H */
