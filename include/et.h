/*
 * et.h -- C ABI of libet: GB300 grain-pair seeded straight-line track finding
 * in nuclear-emulsion views (Ariga & Ariga, "Fast 4pi track reconstruction in
 * nuclear emulsion detectors based on GPU technology", Section 2).
 *
 * Problem (Section 2, Fig. 4).  A view is a 3D cloud of grains (the output of
 * 3D grain recognition).  Every grain pair whose separation lies in the seed
 * window defines a line hypothesis, at any angle (4 pi).  The grains of the
 * whole view lying within the tube radius of that line are counted.  A seed
 * whose count reaches the threshold is a candidate track.  Each grain is then
 * associated with one track only, and the threshold is applied again to the
 * grains that remain.  The survivors get a least-squares line fit, and their
 * start and end points along the line (Fig. 3).
 *
 * Exact semantics implemented here (the paper leaves these open):
 *   - coordinates are int32 in caller units (10 nm in the shipped workloads);
 *   - seeds: unordered pairs {a, b} with seed_min^2 <= |g_b - g_a|^2 < seed_max^2;
 *     the pair is oriented lo -> hi where lo comes first in lexicographic
 *     (x, y, z) order ("canonical rank");
 *   - count(lo, hi) = #{k : |(g_k - g_lo) x (g_hi - g_lo)|^2 <= tube_r^2 |g_hi - g_lo|^2}
 *     over all grains of the view (infinite line, closed tube, seed grains
 *     included), computed in exact integer arithmetic;
 *   - candidates: count >= min_hits;
 *   - exclusive association: the result equals visiting the candidates in the
 *     order (count descending, rank of lo ascending, rank of hi ascending) and
 *     accepting a candidate iff at least min_hits of its tube grains are not
 *     yet used by an earlier accepted track; the accepted track owns exactly
 *     those grains;
 *   - fit (not in the paper): orthogonal least squares in FP32 -- centroid c,
 *     unit principal axis u of the scatter matrix (cyclic Jacobi), oriented so
 *     that u . (g_hi - g_lo) > 0, and tmin / tmax = min / max of (g - c) . u
 *     over the members.  The segment runs from c + tmin u to c + tmax u.
 *
 * Results are bit-identical to a plain CPU evaluation of the definition for
 * everything but the fit; they do not depend on the input order of the grains
 * (up to relabelling) nor on any tuning choice.
 *
 * Errors.  Every call returns an et_status; ET_OK is 0, failures are negative.
 * No exception crosses this boundary and there is no CPU fallback: without a
 * CUDA device the context cannot be created.  et_last_error() returns a
 * thread-local, human-readable description of the last failure on the calling
 * thread.
 */
#ifndef ET_H
#define ET_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ET_ABI_VERSION 3

typedef int32_t et_status;
#define ET_OK                    0
#define ET_ERR_INVALID_ARG      -1  /* null pointer, bad size or parameter */
#define ET_ERR_OUT_OF_RANGE     -2  /* a coordinate outside [0, extent) */
#define ET_ERR_DUPLICATE_GRAIN  -3  /* two grains with identical coordinates in one view */
#define ET_ERR_PRECONDITION     -4  /* parameters break an integer bound of the exact test */
#define ET_ERR_CAPACITY         -5  /* a caller buffer is too small; required sizes returned */
#define ET_ERR_OOM              -6  /* device memory could not be allocated */
#define ET_ERR_BUSY             -7  /* server memory budget or queue full; retry later */
#define ET_ERR_TIMEOUT          -8  /* a bounded device-side wait ran out; results invalid */
#define ET_ERR_CUDA             -9  /* a CUDA runtime call failed */
#define ET_ERR_NOT_READY       -10  /* nothing has been computed yet */

/* Variants (et_params.flags).  The default (0) is the sequential greedy
 * association described at the top of this file.
 *
 * ET_FLAG_SINGLE_PASS -- the other reading of "each grain is exclusively
 *   associated with one track" (Section 2): every grain of a candidate's tube
 *   goes to the best candidate (candidate order above) whose tube holds it, in
 *   one pass; a candidate becomes a track iff at least min_hits grains went to
 *   it, and owns exactly those.  A grain whose best candidate is rejected stays
 *   unassigned.
 * ET_FLAG_ANGLE_CUT -- the grain-count cut against background of Section 3
 *   (Fig. 9c: larger-angle tracks have more grains): a track is kept iff
 *       nhits >= cut_base + cut_slope * min(tan theta, cut_tan_max),
 *   theta being the angle of its seed vector w = g_hi - g_lo to the z axis
 *   (tan theta = sqrt(w_x^2 + w_y^2) / |w_z|, infinite for w_z = 0), decided
 *   in exact integer arithmetic.  Dropped tracks keep their grains (the cut
 *   selects tracks; it does not re-associate grains). */
#define ET_FLAG_SINGLE_PASS 1u
#define ET_FLAG_ANGLE_CUT   2u

/* Tracking parameters (Section 2).  Distances in coordinate units.
 * extent[k] > 0: grains must lie in [0, extent[k]).  Limits enforced:
 *   extent[k] <= 2^21, views of at most 2^21 - 1 grains,
 *   0 <= seed_min <= seed_max, 1 <= seed_max, 0 <= tube_r <= 2^20, 1 <= min_hits,
 *   (extent[a] + extent[b]) * seed_max < 2^31 for every pair of axes a != b
 *   (so every cross-product component is an exact int32) and
 *   3 tube_r^2 seed_max^2 < 2^63 (so the tube bound r^2 |w|^2 is an exact
 *   int64), else ET_ERR_PRECONDITION.  flags: a combination of the ET_FLAG_* bits above.
 *   With ET_FLAG_ANGLE_CUT: 0 <= cut_base <= 2^21, 0 <= cut_slope <= 2^20,
 *   0 <= cut_tan_max <= 1024 (cut fields are ignored without it); reserved = 0. */
typedef struct {
    int32_t extent[3];
    int32_t seed_min, seed_max;
    int32_t tube_r;
    int32_t min_hits;
    uint32_t flags;
    int32_t cut_base;       /* grains */
    int32_t cut_slope;      /* grains per unit of tan theta */
    int32_t cut_tan_max;    /* tan theta above this counts as this */
    int32_t reserved;
} et_params;

/* Optional tuning.  Zero fields mean "choose automatically".  Results never
 * depend on these values, only the speed does. */
typedef struct {
    int32_t cell[3];        /* cell-list edge per axis, coordinate units; 0: automatic
                               (s0 * (0.22, 1.1, 1.1), s0 the edge of a cube holding 0.35
                               grains at the batch's mean density).  The batch's cell table
                               (views x cells per view) must stay below 2^31 - 1 cells, else
                               loading fails with ET_ERR_INVALID_ARG */
    int32_t ticket_origins; /* origins per work ticket of the seed generator (a warp takes
                               this many consecutive grains as line origins at a time):
                               1, 2 or 4; 0: automatic (2) */
    int32_t row_lists;      /* 1: one cell list, rows along x; 2: also a list with rows
                               along y, used by lines whose |w_y| > |w_x|; 0: automatic (2) */
    int32_t assoc_window;   /* candidates per window of the exclusive association (the
                               rounds run window by window in candidate order); 0: automatic
                               (at least 2^18, at most 128 windows) */
    int32_t wait_polls;     /* 0: default.  Otherwise every bounded device-side wait (the
                               grid barriers of the association, the sorts and the scans;
                               the sorts' look-back) gives up
                               after this many polls and the run fails with ET_ERR_TIMEOUT.
                               Small values make a wait run out on purpose (tests of the
                               timeout path); the next run with 0 is unaffected */
    int32_t reserved;
} et_tuning;

/* One reconstructed track.  seed_i / seed_j are indices into the caller's grain
 * array of the view (seed_i is the lower-rank grain).  count is the seed's tube
 * count (all grains along its line, the candidate's rank key); nhits <= count
 * is the number of grains the track owns after exclusive association.
 * member_offset indexes the member array returned with it; members of one
 * track are ascending grain indices of the view. */
typedef struct {
    int32_t seed_i, seed_j;
    int32_t nhits;
    int32_t view;
    int64_t member_offset;
    float c[3];
    float u[3];
    float tmin, tmax;
    int32_t count;
    int32_t reserved;
} et_track;

/* Counters of the last completed run. */
typedef struct {
    int64_t n_grains;
    int64_t n_seeds;        /* seed hypotheses evaluated */
    int64_t n_tests;        /* tube-membership tests performed (cell cover) */
    int64_t n_hits;         /* sum of tube counts over all seeds */
    int64_t n_candidates;   /* seeds with count >= min_hits */
    int64_t n_members;      /* sum of counts over candidates */
    int64_t n_tracks;       /* accepted tracks */
    int64_t n_track_members;
    int32_t merge_rounds;
    int32_t cell[3];        /* cell edge actually used */
    int32_t kernel_launches;/* kernels one run of the path launches (from its captured graph) */
    int32_t profiled;       /* 1 if stage_ms holds timings of the last run */
    /* with profiling on: CUDA-event time of each stage of the last run, ms:
     * 0 canonical order + cell list, 1 (empty: the seeds are generated inside
     * the tube-count kernel), 2 seeds + tube counts, 3 candidate keys + member
     * lists, 4 merge, 5 output (order, fit, members) */
    float stage_ms[6];
    int64_t n_pair_tests;   /* seed-window tests the seed generator made (grain pairs examined) */
} et_stats;

typedef struct et_ctx et_ctx;
typedef struct et_batch et_batch;
typedef struct et_server et_server;
typedef et_batch et_view;   /* a view is a batch of one */

/* ------------------------------------------------------------------ context */

/* Device memory hooks.  alloc returns a device pointer of at least `bytes`
 * (aligned to 256 bytes) or NULL; free releases it.  Without hooks the library
 * uses cudaMalloc / cudaFree. */
typedef void *(*et_alloc_fn)(size_t bytes, void *user);
typedef void (*et_free_fn)(void *ptr, void *user);

/* Creates a context on CUDA device `device` (made current on the calling
 * thread).  The context owns a stream used when callers pass NULL. */
et_status et_ctx_create(int device, et_ctx **out);
et_status et_ctx_destroy(et_ctx *ctx);
et_status et_ctx_set_allocator(et_ctx *ctx, et_alloc_fn alloc, et_free_fn free_fn, void *user);
/* Number of SMs, for callers sizing their own work. */
et_status et_ctx_info(et_ctx *ctx, int32_t *sm_count, int32_t *cc_major, int32_t *cc_minor);

/* ------------------------------------------------------------------ views (plain form) */

/* Creates a view from n grains (row-major int32 [n][3]) in HOST memory.  The
 * grains are copied; the caller may free them on return.  Validation of the
 * coordinates happens on the device and is reported by et_track_fetch. */
et_status et_view_create(et_ctx *ctx, const int32_t *xyz, int64_t n, const et_params *params,
                         et_view **out);
/* Same, with xyz in DEVICE memory of the context's device.  The grains are
 * copied on the context stream; the caller keeps ownership of xyz. */
et_status et_view_create_device(et_ctx *ctx, const int32_t *d_xyz, int64_t n,
                                const et_params *params, et_view **out);
/* Replaces the grains of an existing view (host memory), reusing its device
 * buffers where they are large enough.  The copy is enqueued on `stream`
 * (NULL = context stream) from the caller's buffer, which must stay valid until
 * the next et_track_fetch on this view returns. */
et_status et_view_load(et_view *view, const int32_t *xyz, int64_t n, void *stream);
et_status et_view_destroy(et_view *view);

/* Enqueues the whole hot path on `stream` (a cudaStream_t; NULL = context
 * stream) and returns without waiting. */
et_status et_track_find(et_view *view, void *stream);

/* Waits for the view's last et_track_find, then copies the tracks (in
 * acceptance order) and their members into caller buffers.  If a buffer is too
 * small, ET_ERR_CAPACITY is returned with *n_tracks / *n_members set to the
 * required sizes; the results stay on the device and the call may be repeated.
 * Device-side overflow of internal buffers is handled here by growing them and
 * running the path again.  Coordinate errors (ET_ERR_OUT_OF_RANGE,
 * ET_ERR_DUPLICATE_GRAIN) and ET_ERR_TIMEOUT surface here. */
et_status et_track_fetch(et_view *view, et_track *tracks, int64_t cap, int64_t *n_tracks,
                         int32_t *members, int64_t member_cap, int64_t *n_members);

/* Per-seed tube counts of the last run: seeds (seed_i, seed_j, count) for every
 * seed hypothesis, in no particular order (parity checks and diagnostics).
 * The view runs the path once more with a per-seed record buffer (no flag or
 * earlier setup needed).  Returns ET_ERR_CAPACITY with *n_seeds = required
 * size if cap is too small.  Also accepts a batch (an et_view is a batch of
 * one): seed_i / seed_j then index the batch's grains back to back, i.e.
 * offsets[v] + the index within view v. */
et_status et_view_seed_counts(et_view *view, int32_t *seed_i, int32_t *seed_j, int32_t *count,
                              int64_t cap, int64_t *n_seeds);

/* ------------------------------------------------------------------ batches */

/* A batch holds many views that share one et_params.  All views are processed
 * by one sequence of launches (persistent kernels with a global work queue),
 * replayed from a CUDA graph when the batch shape repeats. */
et_status et_batch_create(et_ctx *ctx, const et_params *params, et_batch **out);
/* Loads n_views views: xyz holds all grains back to back (int32 [total][3]),
 * view v owning rows [offsets[v], offsets[v+1]).  on_device != 0: xyz is a
 * device pointer (copied device-to-device, async); else host memory (copied
 * async from the caller's buffer, which must stay valid until the next fetch).
 * offsets is always host memory (n_views + 1 entries, offsets[0] = 0). */
et_status et_batch_load(et_batch *b, const int32_t *xyz, const int64_t *offsets, int32_t n_views,
                        int32_t on_device, void *stream);
et_status et_batch_set_tuning(et_batch *b, const et_tuning *tuning);
/* Picks the tuning for the loaded batch by timing the whole path on it: up to
 * max_trials candidate cell shapes derived from the batch's mean grain
 * density (mostly anisotropic, cells along the x rows kept short), each with
 * one cell list and with both lists, then 1, 2 and 4 origins per work ticket
 * for the fastest shape (unless ticket_origins was set); two runs each,
 * CUDA-event timed.  The fastest is kept as the batch's tuning and returned in
 * *chosen (may be NULL), its time per run in *best_ms (may be NULL).
 * Synchronous.  Results never depend on the choice, only the speed does. */
et_status et_batch_autotune(et_batch *b, void *stream, int32_t max_trials, et_tuning *chosen, float *best_ms);
/* Enqueues the path for all loaded views.  use_graph != 0 captures the launch
 * sequence once per batch shape and replays it. */
et_status et_batch_find(et_batch *b, void *stream, int32_t use_graph);
/* Like et_track_fetch for all views: tracks ordered by (view, acceptance
 * order); view_track_offsets (n_views + 1 entries, may be NULL) receives where
 * each view's tracks start.  member_offset of a track indexes `members`. */
et_status et_batch_fetch(et_batch *b, int64_t *view_track_offsets, et_track *tracks, int64_t cap,
                         int64_t *n_tracks, int32_t *members, int64_t member_cap,
                         int64_t *n_members);
et_status et_batch_stats(et_batch *b, et_stats *out);
/* on != 0: record a CUDA event between the stages of every later run (also
 * inside captured graphs) so that et_batch_stats reports stage times. */
et_status et_batch_set_profiling(et_batch *b, int32_t on);
/* Waits for the batch without copying anything back; returns the run status. */
et_status et_batch_sync(et_batch *b);
et_status et_batch_destroy(et_batch *b);

/* ------------------------------------------------------------------ server */

/* A served loop: views are submitted one by one as a scanning microscope
 * emits them, grouped into micro-batches by a worker thread and processed on
 * the device; per-view results are kept until polled.  Two micro-batches
 * alternate (one runs while the next is staged).  mem_budget_bytes bounds the
 * device memory both micro-batches hold together at any time: a micro-batch is
 * admitted only while its planned buffers plus the other one's fit, and a
 * micro-batch whose buffers would have to grow past what the other leaves
 * (after a candidate overflow) fails its views with ET_ERR_OOM.  Host staging
 * memory is not counted. */
typedef struct {
    uint64_t tag;            /* caller's tag from et_server_submit */
    et_status status;
    int32_t n_tracks;
    int64_t n_members;
    int64_t n_grains;
    int64_t t_submit_ns;     /* CLOCK_MONOTONIC timestamps */
    int64_t t_admit_ns;
    int64_t t_done_ns;
} et_result;

/* Counters of a server. */
typedef struct {
    uint64_t budget_bytes;
    uint64_t device_bytes;       /* device memory its micro-batches hold now */
    uint64_t peak_device_bytes;  /* the most they held together at any time */
    int64_t views_done;          /* views whose results were produced */
    int64_t batches;             /* micro-batches run */
    int64_t busy_rejections;     /* submits answered with ET_ERR_BUSY */
    int64_t pending;             /* views queued, not yet admitted */
} et_server_stats;

et_status et_server_create(et_ctx *ctx, const et_params *params, uint64_t mem_budget_bytes,
                           int32_t max_batch_views, et_server **out);
/* Copies the view's grains (host memory) and queues it.  ET_ERR_BUSY if the
 * pending queue is full (back-pressure: retry later) or if the view alone
 * needs more device memory than the budget. */
et_status et_server_submit(et_server *s, const int32_t *xyz, int64_t n, uint64_t tag);
/* Returns up to `max` finished views (oldest first), waiting up to timeout_us
 * microseconds for at least one.  Each result's tracks may be copied with
 * et_server_fetch before the next poll. */
et_status et_server_poll(et_server *s, et_result *out, int32_t max, int32_t *n_done,
                         int32_t timeout_us);
/* Tracks of a result returned by the last et_server_poll, by its tag. */
et_status et_server_fetch(et_server *s, uint64_t tag, et_track *tracks, int64_t cap,
                          int64_t *n_tracks, int32_t *members, int64_t member_cap,
                          int64_t *n_members);
/* Pending-queue length at which et_server_submit answers ET_ERR_BUSY
 * (default 2^20 views; at least 1). */
et_status et_server_set_max_pending(et_server *s, int64_t max_pending);
et_status et_server_get_stats(et_server *s, et_server_stats *out);
et_status et_server_destroy(et_server *s);

/* ------------------------------------------------------------------ no allocation */

/* The paper has no counterpart to this entry point: it exists for callers
 * that cannot call cudaMalloc -- an acquisition loop that must not block on
 * the device-wide synchronisation an allocation can cause, code running in a
 * host function enqueued on a stream (where CUDA calls are not allowed), or
 * an application whose framework has already reserved the free device memory
 * for its own pool.
 *
 * For each pair k (d_pairs[2k], d_pairs[2k+1]: indices into the view's grains)
 * it writes to d_counts[k] the number of grains of the view within tube_r of
 * the line through the two grains -- the same exact count et_view_seed_counts
 * reports for a seed -- or -1 for a pair with an index outside [0, n), two
 * equal indices, two grains at the same coordinates, or grains seed_max or
 * more apart along some axis (the bound under which the exact integer test
 * cannot overflow; every seed of the window lies within it), and -1 for every
 * pair if a coordinate lies outside [0, extent).  d_xyz (int32 [n][3]), d_pairs (int32 [n_pairs][2]) and d_counts
 * (int32 [n_pairs]) are DEVICE memory of the current device, owned by the
 * caller; the work is enqueued on `stream` (NULL = legacy default stream) and
 * the call returns without waiting.
 *
 * Nothing is allocated.  The intermediate cell list lives in one fixed
 * array of about 3 MB (ET_NOALLOC_MAX_GRAINS grains, ET_NOALLOC_MAX_CELLS cells)
 * that every GPU which loads the library keeps until the process exits.  The
 * first call on a device looks up that array's device address; make it
 * before any stream capture (the address is looked up again after a device
 * reset has replaced the device's context).  All calls share the array, so calls whose work
 * overlaps on the GPU race: order them (one stream, or events).  Views larger
 * than ET_NOALLOC_MAX_GRAINS are rejected with ET_ERR_INVALID_ARG. */
#define ET_NOALLOC_MAX_GRAINS 65536
#define ET_NOALLOC_MAX_CELLS 262144
et_status et_tube_count_noalloc(const int32_t *d_xyz, int64_t n, const et_params *params,
                                const int32_t *d_pairs, int64_t n_pairs, int32_t *d_counts, void *stream);

/* ------------------------------------------------------------------ misc */

const char *et_last_error(void);
const char *et_status_string(et_status s);
int32_t et_abi_version(void);

#ifdef __cplusplus
}
#endif
#endif /* ET_H */
