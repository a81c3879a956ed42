/*
 * et_frames.h -- C ABI of libet's image front end: from the raw frames of
 * emulsion views to grains (Ariga & Ariga, "Fast 4pi track reconstruction in
 * nuclear emulsion detectors based on GPU technology", Section 2: filtering
 * and 3D grain recognition, Fig. 2).
 *
 * A view is digitised into `depth` frames of `width` x `height` 8-bit pixels
 * (1280 x 1024 x 40 in the paper); grains are dark in the raw image.
 *
 * Filtering (Section 2).  The pixels of the camera differ in gain, so every
 * pixel (x, y) carries its own gain g (8 bits, 128 = 1.0) and threshold t,
 * and the image is inverted.  The filtered pulse height of a raw value is
 *     f = max(0, min(255, floor(((255 - raw) * g + 64) / 128)) - t).
 * The paper names these three operations without their form; this is the
 * reading implemented here, in exact integer arithmetic.
 *
 * 3D grain recognition (Section 2).  A voxel p with f(p) > grain_threshold
 * defines a grain when no voxel among its 3 x 3 x 3 neighbours (inside the
 * view's stack) beats it: f(q) < f(p) for every neighbour q before p in raster
 * order (frame, row, column) and f(q) <= f(p) for every neighbour after it, so
 * of two equal neighbours the first wins.  The grain's position is the
 * pulse-height centre of mass of that neighbourhood: voxel index i along axis
 * k lies at i * pitch_num[k] / pitch_den[k] coordinate units and, with
 * S = sum f(q) and S_k = sum f(q) q_k over the neighbourhood, the coordinate
 * is S_k * pitch_num[k] / (S * pitch_den[k]) rounded half up.
 *
 * Results are exact (bit-identical to a plain CPU evaluation of these
 * definitions).  Grains of a view come in raster order of the voxel that
 * defines them.  Errors follow et.h: every call returns an et_status, no
 * exception crosses this boundary, and there is no CPU fallback.
 */
#ifndef ET_FRAMES_H
#define ET_FRAMES_H

#include "et.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Camera geometry and recognition threshold.  Limits enforced:
 *   1 <= width <= 4096, 1 <= height <= 4096, 1 <= depth <= 1024;
 *   row_pitch >= width and a multiple of 16 (bytes between consecutive rows
 *   of the raw frames; frames and views follow each other without gaps);
 *   1 <= pitch_num[k], pitch_den[k] <= 65535;  0 <= grain_threshold <= 254;
 *   flags == 0.  Otherwise ET_ERR_INVALID_ARG. */
typedef struct {
    int32_t width, height, depth;
    int32_t row_pitch;
    int32_t pitch_num[3], pitch_den[3];
    int32_t grain_threshold;
    uint32_t flags;
} et_frame_params;

/* Counters of the last completed run. */
typedef struct {
    int64_t n_views;
    int64_t n_voxels;        /* voxels examined: n_views * depth * height * width */
    int64_t n_candidates;    /* voxels with f > grain_threshold */
    int64_t n_grains;
    float kernel_ms;         /* CUDA-event time of the recognition kernel */
    float run_ms;            /* CUDA-event time of the whole run on the device (upload included) */
    int32_t kernel_launches; /* kernels one run launches (recognition, sort passes, gather, scan) */
    int32_t reserved;
} et_frames_stats;

typedef struct et_frames et_frames;

/* Creates a front end for one camera: gain and thr are HOST arrays of
 * height x width bytes (row-major), copied.  Allocates the device tables; the
 * per-run buffers grow on demand. */
et_status et_frames_create(et_ctx *ctx, const et_frame_params *params, const uint8_t *gain,
                           const uint8_t *thr, et_frames **out);
/* Replaces the per-pixel calibration (same layout as in et_frames_create). */
et_status et_frames_set_calibration(et_frames *fr, const uint8_t *gain, const uint8_t *thr);

/* Enqueues filtering and grain recognition of n_views >= 1 views on `stream`
 * (NULL = context stream) and returns without waiting.  raw holds the views
 * back to back, each depth x height x row_pitch bytes.  on_device != 0: raw is
 * device memory of the context's device, read in place (keep it unchanged
 * until the next et_frames_fetch / et_frames_sync returns; its address must be
 * 16-byte aligned); else host memory, copied asynchronously into a device
 * buffer (page-locked memory makes the copy asynchronous; keep it valid until
 * the next fetch or sync). */
et_status et_frames_run(et_frames *fr, const uint8_t *raw, int32_t n_views, int32_t on_device,
                        void *stream);

/* Waits for the last run; returns its status.  Output overflow is handled
 * here by growing the grain buffer and running again. */
et_status et_frames_sync(et_frames *fr);

/* Waits for the last run and copies its grains to host buffers:
 * view_offsets (n_views + 1 entries, may be NULL): where each view's grains
 * start; xyz (int32 [n][3]) and pulse (int32 [n], may be NULL: the sum of the
 * neighbourhood's pulse heights).  ET_ERR_CAPACITY with *n_grains set if cap
 * is too small; the call may be repeated. */
et_status et_frames_fetch(et_frames *fr, int64_t *view_offsets, int32_t *xyz, int32_t *pulse, int64_t cap,
                          int64_t *n_grains);

/* Waits for the last run and loads its grains into a batch, one view per
 * frame stack, device to device on `stream` (NULL = context stream); the batch
 * must have been created with the same context.  Then et_batch_find runs the
 * track finding on them.  The grain coordinates must lie inside the batch's
 * et_params extent: with voxel pitch num/den they are at most
 * ((n - 1) * num + den / 2) / den along an axis of n voxels. */
et_status et_frames_to_batch(et_frames *fr, et_batch *batch, void *stream);

et_status et_frames_stats_get(et_frames *fr, et_frames_stats *out);
et_status et_frames_destroy(et_frames *fr);

#ifdef __cplusplus
}
#endif
#endif /* ET_FRAMES_H */
