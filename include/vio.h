/*
 * vio.h -- C ABI of the GB300 stereo visual frontend (libvio.so).
 *
 * Method: VkVIO, "Cross-platform GPU Acceleration for Visual-Inertial
 * Odometry with Vulkan" (arxiv 2609.30459), Sec. III: per frame, an image
 * pyramid (Sec. III-C), grid-cell FAST-9 detection (Sec. III-D) and
 * patch-based inverse-compositional KLT tracking, temporal and across the
 * stereo pair, with a forward-backward check (Sec. III-E).
 *
 * Conventions for every call:
 *  - Pointers named d_* are DEVICE pointers owned by the caller; the library
 *    never frees or retains them past the call's completion on the stream.
 *    Host structs passed by pointer are read during the call only.
 *  - Calls are asynchronous on the given cudaStream_t (passed as void*;
 *    NULL = the legacy default stream). They enqueue kernels and return; no
 *    host synchronisation and no allocation happen outside *_create.
 *  - Arguments are validated on the host before anything is enqueued. A call
 *    that returns non-zero has enqueued nothing, except VIO_ERR_CUDA, which
 *    reports a launch error from the CUDA runtime.
 *  - Images are uint8, row-major, with a row pitch in bytes. Pixel centres
 *    are at integer coordinates; level-l coordinates are level-0 coordinates
 *    divided by 2^l. Keypoints are float32 (x, y) in level-0 pixels.
 *  - Batches: calls work on n_images images of one size at fixed strides
 *    (vio_pyr_batch), e.g. the two cameras of a stereo pair, or many frames.
 */
#ifndef VIO_H_
#define VIO_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status -- */
typedef int32_t vio_status;
enum {
  VIO_OK = 0,
  VIO_ERR_INVALID_ARG = 1, /* a pointer, size or parameter is invalid      */
  VIO_ERR_CUDA = 2,        /* the CUDA runtime reported an error           */
  VIO_ERR_OOM = 3,         /* device allocation failed in *_create          */
  VIO_ERR_TIMEOUT = 4,     /* a bounded wait expired (device status word, or
                              the serving loop's host timeout)              */
  VIO_ERR_UNSUPPORTED = 5  /* valid but outside what this build handles    */
};

/* Per-keypoint track status (uint8). */
enum {
  VIO_TRACK_OK = 0,
  VIO_TRACK_OOB_TEMPLATE = 1, /* level-0 template leaves the source image    */
  VIO_TRACK_OOB_WARP = 2,     /* a warped sample leaves the target image     */
  VIO_TRACK_DEGENERATE_H = 3, /* level-0 Hessian not positive definite       */
  VIO_TRACK_ZERO_MEAN = 4,    /* patch mean <= 0 (Eq. 4 undefined)           */
  VIO_TRACK_FB_FAIL = 5,      /* forward-backward distance above threshold   */
  VIO_TRACK_NAN = 6,          /* non-finite Gauss-Newton increment           */
  VIO_TRACK_EMPTY = 255       /* slot holds no keypoint                      */
};

#define VIO_MAX_LEVELS 8
#define VIO_MAX_THRESHOLDS 8
#define VIO_MAX_K 8

/* ---------------------------------------------------------------- params -- */
/* Frontend parameters. Defaults (vio_params_default) follow the paper:
 * threshold sequence <40,20,10,5> and k = 1 (Sec. III-D), 5 Gauss-Newton
 * iterations per level (Sec. III-E), 50 px cells (Sec. IV-D). Values the
 * paper leaves open: 4 levels, round-to-nearest pyramid (Eq. 1), pattern 0,
 * forward-backward threshold 0.2 px, detection border 9 px (the level-0
 * reach of the tracking template), selection VIO_SELECT_WARP_MAX. */
typedef struct {
  int32_t n_levels;                      /* pyramid levels incl. level 0, 1..8 */
  int32_t round_mode;                    /* 0 = nearest (Eq. 1), 1 = floor (Eq. 3) */
  int32_t gn_iters;                      /* Gauss-Newton iterations per level  */
  int32_t pattern_id;                    /* 0 = the 52-point odd lattice       */
  int32_t cell_w, cell_h;                /* detection cell size, level-0 px    */
  int32_t k_per_cell;                    /* keypoints per cell, 1..VIO_MAX_K   */
  int32_t n_thresholds;                  /* 1..VIO_MAX_THRESHOLDS              */
  int32_t thresholds[VIO_MAX_THRESHOLDS];/* descending FAST thresholds, >= 0   */
  int32_t detect_border;                 /* candidates need b <= x <= w-1-b    */
  float fb_max_dist;                     /* forward-backward threshold, px     */
  int32_t select_mode;                   /* per-cell top-k, VIO_SELECT_*       */
} vio_params;

/* How each cell's k strongest maxima are picked (Sec. III-D describes a
 * bitonic k-sort per workgroup and an atomic-maximum variant for one
 * keypoint per cell). Candidates carry unique packed keys (score << 32 |
 * ~(y * w + x)), so every mode gives the same keypoints bit for bit:
 *   VIO_SELECT_WARP_MAX: k rounds of a warp-wide maximum (default);
 *   VIO_SELECT_BITONIC:  a bitonic sort of each warp's candidate keys;
 *   VIO_SELECT_ATOMIC:   a 64-bit atomic maximum per cell, k = 1 only
 *                        (other k: VIO_ERR_INVALID_ARG). */
enum { VIO_SELECT_WARP_MAX = 0, VIO_SELECT_BITONIC = 1, VIO_SELECT_ATOMIC = 2 };

void vio_params_default(vio_params* p);

/* ------------------------------------------------------------ pyramids -- */
/* Geometry of one image's pyramid (Sec. III-C). Level 0 is the caller's
 * frame (pitch level0_pitch); levels 1..n-1 are packed in one caller buffer
 * ("upper buffer") at offset[l], each with a 128-byte-aligned pitch. Level
 * sizes: w_{l+1} = floor(w_l / 2), h_{l+1} = floor(h_l / 2). */
typedef struct {
  int32_t n_levels;
  int32_t w[VIO_MAX_LEVELS], h[VIO_MAX_LEVELS], pitch[VIO_MAX_LEVELS];
  int64_t offset[VIO_MAX_LEVELS]; /* byte offset of level l >= 1 in the upper buffer */
  int64_t upper_bytes;            /* size of the upper buffer, multiple of 256 */
} vio_pyr_layout;

/* Fills *out for a w x h image with n_levels levels. Needs every level at
 * least 1x1 and level0_pitch >= w. */
vio_status vio_pyr_layout_make(int32_t w, int32_t h, int32_t n_levels, int32_t level0_pitch,
                               vio_pyr_layout* out);

/* n_images pyramids of one layout: image i has level 0 at
 * d_level0 + i * level0_stride and its upper buffer at
 * d_upper + i * upper_stride (strides in bytes, upper_stride >= upper_bytes
 * and a multiple of 16). */
typedef struct {
  const uint8_t* d_level0;
  int64_t level0_stride;
  uint8_t* d_upper;
  int64_t upper_stride;
  int32_t n_images;
} vio_pyr_batch;

/* ------------------------------------------------------------- context -- */
typedef struct vio_ctx vio_ctx;

/* Allocates the scratch the calls below need for images up to max_w x
 * max_h and batches up to max_images. The only allocating calls are
 * vio_ctx_create and vio_frontend_create. Cells whose per-block shared
 * memory would exceed 200 KiB (about 125 x 125 px) return
 * VIO_ERR_UNSUPPORTED. */
vio_status vio_ctx_create(vio_ctx** ctx, const vio_params* p, int32_t max_w, int32_t max_h,
                          int32_t max_images);
vio_status vio_ctx_destroy(vio_ctx* ctx);
const char* vio_status_string(vio_status s);

/* Device-side errors. Arguments are checked on the host before anything is
 * enqueued; what can only go wrong on the device (a bounded wait that gave
 * up) is recorded in the context's device status word: VIO_OK, or the first
 * such error since the word was last cleared.
 *   vio_ctx_sync:   enqueues a read and a clear of the word on `stream`, waits
 *                   for the stream, and stores the word in *device_status;
 *                   returns VIO_ERR_CUDA if the stream reported an error.
 *   vio_last_error: reads the word (a blocking copy) without clearing it and
 *                   returns it (VIO_ERR_CUDA if the read failed). */
vio_status vio_ctx_sync(vio_ctx* ctx, void* stream, vio_status* device_status);
vio_status vio_last_error(vio_ctx* ctx);

/* A bounded wait on the device: enqueues on `stream` a wait until the int32
 * at d_flag (device memory, or host memory mapped into the device, written by
 * another stream or by the host) equals `value`. Work after it on the stream
 * starts once the flag is set, or once timeout_ns (0 .. 2 s) has passed: the
 * wait then records VIO_ERR_TIMEOUT in the context's status word and ends, so
 * the context and the stream stay usable. The paper has no counterpart (its
 * host waits on a fence, Sec. III-B). */
vio_status vio_wait_flag(vio_ctx* ctx, const int32_t* d_flag, int32_t value, int64_t timeout_ns,
                         void* stream);

/* --------------------------------------------------------------- stages -- */

/* Sec. III-C, Eq. 1-3: builds levels 1..n-1 of every pyramid of the batch
 * from its level 0: a separable 5x5 binomial [1,4,6,4,1] filter, 2:1
 * subsampling, integer arithmetic, rounding per p->round_mode, edges
 * clamped. Reads level 0, writes the upper buffers. */
vio_status vio_pyramid_build(vio_ctx* ctx, const vio_pyr_layout* layout,
                             const vio_pyr_batch* batch, void* stream);

/* Sec. III-D: the FAST-9 score of every pixel of one image: the largest
 * integer tau >= 0 for which 9 contiguous pixels of the 16-pixel radius-3
 * Bresenham circle are all brighter than I(p)+tau or all darker than
 * I(p)-tau; -1 where there is none or the circle leaves the image.
 * d_score: w*h int16, row-major, pitch w elements. */
vio_status vio_fast_scores(const uint8_t* d_img, int32_t w, int32_t h, int32_t pitch,
                           int16_t* d_score, void* stream);

/* Sec. III-D: grid-cell detection on level 0 of every image of the batch.
 * Cells are the full cell_w x cell_h cells of a grid anchored at (0,0)
 * (gx = w / cell_w by gy = h / cell_h). Per cell, for the thresholds in
 * turn: corners with score >= T, strict 3x3 local maxima (compared with all
 * 8 image neighbours), the strongest k_eff = k - occupancy[cell] of them,
 * stopping at the first threshold that yields k_eff; ties ordered by
 * (score desc, y asc, x asc). Equivalent one-pass form is used.
 *   d_occupancy: per image gx*gy uint8 counts of existing tracks (raster
 *                order, image stride gx*gy), or NULL for none.
 *   d_mask:      per image w*h uint8, 0 = pixel excluded, image stride
 *                mask_stride, row pitch w; or NULL.
 *   d_kp, d_score: per image `capacity` slots (image stride capacity): the
 *                keypoints in cell raster order, then by rank; float2 (x,y)
 *                and int16 score.
 *   d_count:     per image int32, the number written (<= capacity).
 * Uses the context's scratch: calls on one context must not overlap. */
vio_status vio_detect_grid(vio_ctx* ctx, const vio_pyr_layout* layout,
                           const vio_pyr_batch* batch, const uint8_t* d_occupancy,
                           const uint8_t* d_mask, int64_t mask_stride, float* d_kp,
                           int16_t* d_score, int32_t* d_count, int32_t capacity, void* stream);

/* Sec. III-C and III-D together: vio_pyramid_build and vio_detect_grid of the
 * same batch, for throughput over many images: per chunk of images whose
 * level 0 fits in half the L2, the pyramid launches and then the detection
 * launches, so level 0 comes from DRAM once. Arguments and results as the two
 * calls. The pyramid needs n_levels == the context's n_levels. */
vio_status vio_pyramid_detect(vio_ctx* ctx, const vio_pyr_layout* layout,
                              const vio_pyr_batch* batch, const uint8_t* d_occupancy,
                              const uint8_t* d_mask, int64_t mask_stride, float* d_kp,
                              int16_t* d_score, int32_t* d_count, int32_t capacity, void* stream);

/* Detection without any device allocation. The paper has no counterpart:
 * this is a convenience for callers that cannot call cudaMalloc -- code
 * inside a pre-sized memory pool or a budget that forbids new allocations,
 * plugins whose host runtime owns all device memory, real-time loops where an
 * allocation (which may synchronise the device) is not allowed. It computes
 * exactly what vio_detect_grid computes, with the parameters passed directly
 * instead of through a vio_ctx (creating a context allocates).
 *   Scratch: a fixed array inside the library image, per device, sized for
 *   VIO_NOALLOC_MAX_CELL_SLOTS cell slots (8 + 4 bytes each, 768 KiB), held
 *   by every GPU that loads the library until the process exits. A call needs
 *   n_images * cells * k_per_cell slots and n_images * cells counts, each at
 *   most VIO_NOALLOC_MAX_CELL_SLOTS; larger calls return VIO_ERR_UNSUPPORTED.
 *   Set-up: the first call on a device looks up the array's device address
 *   (cudaGetSymbolAddress, with that device current); make it before any
 *   stream capture. Later calls on that device reuse the address.
 *   Sharing: all calls use the same array, which keeps the last call's
 *   contents; each call writes every entry it reads. Calls that overlap on
 *   the GPU race on the array: order them (one stream, or events).
 * Other arguments, layouts and results as vio_detect_grid. */
#define VIO_NOALLOC_MAX_CELL_SLOTS 65536
vio_status vio_detect_grid_noalloc(const vio_params* p, const vio_pyr_layout* layout,
                                   const vio_pyr_batch* batch, const uint8_t* d_occupancy,
                                   const uint8_t* d_mask, int64_t mask_stride, float* d_kp,
                                   int16_t* d_score, int32_t* d_count, int32_t capacity,
                                   void* stream);

/* Flags of vio_track_patches: VIO_TRACK_FORWARD or VIO_TRACK_WITH_FB, or'ed
 * with VIO_TRACK_FROM_LEVEL(l) to track over levels l..0 only (both
 * directions) instead of the whole pyramid; l < n_levels. */
enum { VIO_TRACK_FORWARD = 0, VIO_TRACK_WITH_FB = 1 };
#define VIO_TRACK_FROM_LEVEL(l) (((l) + 1) << 4)

/* Sec. III-E, Eq. 4-5: pyramidal inverse-compositional KLT of 52-point
 * patches with an SE(2) warp (t_x, t_y, theta), coarse to fine, gn_iters
 * Gauss-Newton steps per level, from pyramid src[i] to dst[i]. The warp maps
 * pattern offset x to R(theta) x + t; t is the keypoint's position in the
 * target. One warp of 32 threads tracks one keypoint.
 *   d_pts:    per image `capacity` float2 source positions (image stride
 *             capacity), level-0 px.
 *   d_init:   per keypoint float3 starting warp (t_x, t_y, theta), same
 *             indexing, or NULL for the identity start t = p, theta = 0.
 *   d_count:  per image int32 number of valid keypoints (<= capacity), or
 *             NULL for `capacity` each.
 *   d_out:    per keypoint float3 forward result (t_x, t_y, theta), level 0.
 *   d_status: per keypoint uint8 VIO_TRACK_* status; slots >= count get
 *             VIO_TRACK_EMPTY.
 *   d_fb_dist: per keypoint float forward-backward distance (NaN if not
 *             computed), or NULL.
 *   d_last_step: per keypoint float, how far the forward pass's last
 *             Gauss-Newton step at level 0 moved the pattern (|dx| + |dy| +
 *             7.62 |dtheta|, level-0 px: a convergence measure; NaN where the
 *             forward pass failed), or NULL.
 * flags = VIO_TRACK_WITH_FB also runs the backward pass (template rebuilt on
 * the target at the forward result, warp started at the forward estimate's
 * inverse) and marks VIO_TRACK_FB_FAIL when the returned position is more
 * than fb_max_dist from the original. */
vio_status vio_track_patches(vio_ctx* ctx, const vio_pyr_layout* layout,
                             const vio_pyr_batch* src, const vio_pyr_batch* dst,
                             const float* d_pts, const float* d_init, const int32_t* d_count,
                             int32_t capacity, int32_t flags, float* d_out, uint8_t* d_status,
                             float* d_fb_dist, float* d_last_step, void* stream);

/* Sec. III-E cross-camera matching: vio_track_patches with VIO_TRACK_WITH_FB
 * from cam0 pyramids (src) to cam1 pyramids (dst) at the same time step.
 * d_match: per keypoint float2 position in cam1. */
vio_status vio_stereo_match(vio_ctx* ctx, const vio_pyr_layout* layout,
                            const vio_pyr_batch* cam0, const vio_pyr_batch* cam1,
                            const float* d_pts, const float* d_init, const int32_t* d_count,
                            int32_t capacity, float* d_match, uint8_t* d_status,
                            float* d_fb_dist, void* stream);

/* Sec. III-E cross-camera matching for rigs of more than two cameras (the
 * paper's four-camera runs, Sec. IV-A): the keypoints of one source image
 * (src: a batch of one pyramid, e.g. camera 0 of a rig) are tracked with the
 * forward-backward check into each of the dst->n_images target pyramids of
 * the same time step (the rig's other cameras).
 *   d_pts, d_count: the source keypoints (capacity float2) and their count
 *                   (one int32, or NULL for `capacity`);
 *   d_init:   per target and keypoint float3 start (target-major:
 *             n_targets x capacity), e.g. from vio_predict_warp with each
 *             target's extrinsics, or NULL for the identity start;
 *   d_match:  per target and keypoint float2 position in that target,
 *             d_status and d_fb_dist (may be NULL) likewise; slots >= count
 *             get VIO_TRACK_EMPTY. */
vio_status vio_match_cameras(vio_ctx* ctx, const vio_pyr_layout* layout,
                             const vio_pyr_batch* src, const vio_pyr_batch* dst,
                             const float* d_pts, const float* d_init, const int32_t* d_count,
                             int32_t capacity, float* d_match, uint8_t* d_status,
                             float* d_fb_dist, void* stream);

/* Sec. III-E forward-backward check, for callers that run the backward pass
 * themselves: d_back[i] is the backward result (float3) of keypoint d_orig[i]
 * (float2). Where d_status[i] is VIO_TRACK_OK on entry, writes the distance
 * |t_back - orig| to d_dist[i] (if non-NULL) and sets VIO_TRACK_FB_FAIL when
 * it exceeds max_dist. Other statuses are left as they are. Indexing as in
 * vio_track_patches (n_images x capacity, counts from d_count or all). */
vio_status vio_fb_check(const float* d_orig, const float* d_back, const int32_t* d_count,
                        int32_t capacity, int32_t n_images, float max_dist, uint8_t* d_status,
                        float* d_dist, void* stream);

/* Sec. III-E, the start of a track: the warp begins where the sample pattern
 * lands in the target image when it is carried there by the camera model, the
 * predicted pose and the keypoint's inverse depth. Pinhole cameras; the
 * pose maps points of the source camera into the target camera,
 * P' = R P + t (R row-major).
 * For keypoint u with inverse depth rho: P = (1 / rho) K_src^-1 [u, 1], and
 * u' = the projection of R P + t through K_dst. Each of the 52 pattern points
 * u + x_i is projected the same way at the keypoint's inverse depth (a
 * fronto-parallel patch) to y_i. The start warp is t = u' and theta = the
 * angle of the least-squares rotation from the offsets x_i to y_i - u'
 * (atan2 of sum x_i x (y_i - u') over sum x_i . (y_i - u')).
 *   d_pose:      per image one vio_pose (device memory), e.g. the predicted
 *                motion between the frames of each stream, or the stereo
 *                extrinsics;
 *   d_pts:       per image `capacity` float2 source positions (level-0 px);
 *   d_inv_depth: per keypoint float, same indexing (1 / depth in the source
 *                camera);
 *   d_count:     per image int32 counts, or NULL for `capacity` each;
 *   d_init:      per keypoint float3 (t_x, t_y, theta), the d_init of
 *                vio_track_patches / vio_stereo_match;
 *   d_valid:     per keypoint uint8, 1 where the prediction exists, or NULL.
 * A keypoint with rho <= 0, or whose point or a pattern point is not in front
 * of the target camera, gets the identity start (t = u, theta = 0) and
 * valid 0; slots >= count are not written (valid 0). Invalid intrinsics
 * (fx, fy <= 0) return VIO_ERR_INVALID_ARG. */
typedef struct {
  float fx, fy, cx, cy;
} vio_pinhole;
typedef struct {
  float R[9];
  float t[3];
} vio_pose;

vio_status vio_predict_warp(const vio_pinhole* k_src, const vio_pinhole* k_dst,
                            const vio_pose* d_pose, const float* d_pts, const float* d_inv_depth,
                            const int32_t* d_count, int32_t capacity, int32_t n_images,
                            float* d_init, uint8_t* d_valid, void* stream);

/* ------------------------------------------------------------- frontend -- */
/* The per-frame frontend of Sec. III-B for n_streams independent stereo
 * streams of one size: pyramid of both cameras, temporal tracking of every
 * camera's keypoints with the forward-backward check, detection on camera 0
 * with the cells of surviving tracks counted against k, and stereo matching
 * of the new keypoints into camera 1. State (keypoint lists, ids, pyramids)
 * stays on the device between steps. */
typedef struct vio_frontend vio_frontend;

/* capacity: keypoint slots per camera per stream (gx*gy*k <= capacity <= 32767). */
vio_status vio_frontend_create(vio_frontend** fe, const vio_params* p, int32_t w, int32_t h,
                               int32_t n_streams, int32_t capacity);
vio_status vio_frontend_destroy(vio_frontend* fe);

/* One frame for every stream. d_frames: level-0 images, stream s camera c at
 * d_frames + (2*s + c) * frame_stride, row pitch `pitch`. The buffer is read
 * again by the NEXT step (as the previous frame): keep it unchanged until
 * that step has run. The first step after create or reset only detects. */
vio_status vio_frontend_step(vio_frontend* fe, const uint8_t* d_frames, int32_t pitch,
                             int64_t frame_stride, void* stream);

/* n_steps consecutive steps over frames already in device memory: step i
 * reads d_frames + i * step_stride (same layout as vio_frontend_step). One
 * call enqueues every step (no host work between frames); the usual keep-alive
 * rule applies to the last frame. Without stage timing the steps are
 * pipelined on the frontend's own streams (the pyramids and detection of
 * frame i beside the tracking of frame i-1); they follow the work already on
 * `stream`, and `stream` waits for the last of them. */
vio_status vio_frontend_run(vio_frontend* fe, const uint8_t* d_frames, int32_t pitch,
                            int64_t frame_stride, int64_t step_stride, int32_t n_steps,
                            void* stream);

/* Forget all tracks (next step starts fresh). Enqueued on `stream`. */
vio_status vio_frontend_reset(vio_frontend* fe, void* stream);

/* One step from and to host memory: copies the n_streams stereo frames from
 * h_frames (pinned host memory, the layout of vio_frontend_step) into the
 * caller's device buffer d_frames (kept alive until the next step has run),
 * runs the step, and copies the outputs into the caller's pinned host
 * buffers: track positions, ids and counts of every (stream, camera) list
 * (2 * n_streams * capacity float2 / int32, 2 * n_streams int32; list of
 * stream s camera c at slot (2 s + c) * capacity) and the new detections
 * (n_streams * capacity float2, n_streams int32). All enqueued on `stream`:
 * the host buffers hold the step's results once the stream has passed it. */
vio_status vio_frontend_step_host(vio_frontend* fe, const uint8_t* h_frames, uint8_t* d_frames,
                                  int32_t pitch, int64_t frame_stride, float* h_track_xy,
                                  int32_t* h_track_id, int32_t* h_track_count, float* h_new_xy,
                                  int32_t* h_new_count, void* stream);

/* The same step, pipelined across calls: the upload, pyramids and detection
 * of this step run on the frontend's own low-priority stream beside the
 * tracking of the previous step, the rest on its own high-priority stream,
 * and `done_event` (a cudaEvent_t of the caller, may be NULL) is recorded
 * when the host buffers hold this step's results. The call orders itself
 * after the frontend's own earlier work, and after work the frontend's other
 * calls put on a caller's stream (those in turn wait for the pipelined
 * steps), but not after other work on any caller stream: upload nothing the
 * step reads on another stream without synchronising first. d_frames must
 * stay untouched until done_event of the next step (which reads it as the
 * previous frame). Not with stage timing (VIO_ERR_UNSUPPORTED). */
vio_status vio_frontend_step_host_async(vio_frontend* fe, const uint8_t* h_frames,
                                        uint8_t* d_frames, int32_t pitch, int64_t frame_stride,
                                        float* h_track_xy, int32_t* h_track_id,
                                        int32_t* h_track_count, float* h_new_xy,
                                        int32_t* h_new_count, void* done_event);

/* Device views of the frontend's outputs after the last step, per stream s
 * and camera c at slot base (2*s + c) * capacity:
 *   tracks:  float2 positions, int32 ids, uint8 status (VIO_TRACK_OK for a
 *            live track), int32 counts per (stream, camera) -- TR_t;
 *   new:     per stream, float2 positions and int32 count of the keypoints
 *            detected this step on camera 0 (slot base s * capacity) --
 *            DET_t.
 * The pointers stay valid until destroy; their contents change with every
 * step. */
typedef struct {
  const float* d_track_xy;
  const int32_t* d_track_id;
  const uint8_t* d_track_status;
  const int32_t* d_track_count;
  const float* d_new_xy;
  const int32_t* d_new_count;
  int32_t capacity;
  int32_t n_streams;
} vio_frontend_view;

vio_status vio_frontend_get_view(vio_frontend* fe, vio_frontend_view* out);

/* Number of kernels one vio_frontend_step enqueues (for launch accounting). */
int32_t vio_frontend_launches_per_step(const vio_frontend* fe);

/* Launch shapes of the frontend's steps (vio_batch_tune, defined with the
 * batch below; stereo_after_select must be 0: the frontend keeps the
 * speculative order). Default {128, 0, 0, 0, 256}. Results do not depend on
 * it. A host call between steps. */
struct vio_batch_tune_s;
vio_status vio_frontend_set_tune(vio_frontend* fe, const struct vio_batch_tune_s* t);

/* Stage timing (the paper's per-stage GPU timestamps, Sec. IV-B, Fig. 5).
 * enable: 0 off; 1: every step records CUDA events on its stream at the
 * stage boundaries; 2: only its first and last event (a step's latency with
 * its launches as in an untimed step: events between launches break the
 * overlap of a programmatic dependent with its predecessor; stage_ms then
 * stays 0 for those steps); other values VIO_ERR_INVALID_ARG. Stages: 0
 * pyramid levels 1-4 and the per-cell detection candidates (one launch), 1
 * deeper pyramid levels, 2 learned flow proposals (when the initializer is
 * on), 3 temporal tracking and stereo matching (one launch), 4 finalisation
 * (survivors, per-cell selection, appends).
 * vio_frontend_read_timing waits for the recorded events, adds each stage's
 * elapsed milliseconds into stage_ms[0..VIO_N_STAGES-1] (overwritten), stores
 * the number of timed steps in *n_steps and clears the record. Enabling,
 * disabling and reading are host calls. */
enum { VIO_STAGE_FRONT = 0, VIO_STAGE_PYRAMID_UPPER, VIO_STAGE_INITNET, VIO_STAGE_TRACK,
       VIO_STAGE_FINALIZE, VIO_N_STAGES };
vio_status vio_frontend_set_timing(vio_frontend* fe, int32_t enable);
/* step_ms (may be NULL): per timed step, the time from its first to its last
 * event, for up to step_ms_cap steps in order. */
vio_status vio_frontend_read_timing(vio_frontend* fe, double* stage_ms, int64_t* n_steps,
                                    float* step_ms, int64_t step_ms_cap);

/* Per-step counters, written on the device by every step into a ring of
 * VIO_STATS_RING entries (entry = step index mod the ring size), per stream,
 * VIO_N_STATS int32 values: tracks attempted on cam0 and cam1, tracks that
 * survived on cam0 and cam1, new detections, successful stereo matches of the
 * new detections, detection candidates stereo-matched (every cell's top-k is
 * matched while temporal tracking runs; the selection uses a subset), and
 * surviving tracks (both cameras) that were tracked from the learned
 * initializer's proposal rather than by the plain fallback.
 * vio_frontend_read_stats copies the whole ring to host_out (blocking; size
 * VIO_STATS_RING * n_streams * VIO_N_STATS) and returns the number of steps
 * run since create in *n_steps. */
#define VIO_STATS_RING 4096
enum { VIO_STAT_TRK0 = 0, VIO_STAT_TRK1, VIO_STAT_OK0, VIO_STAT_OK1, VIO_STAT_NEW,
       VIO_STAT_MATCHED, VIO_STAT_CAND, VIO_STAT_LEARNED, VIO_N_STATS };
vio_status vio_frontend_read_stats(vio_frontend* fe, int32_t* host_out, int64_t* n_steps);

/* Learned start of temporal tracking (an addition; the paper starts from a
 * camera-model prediction, Sec. III-E). When on, every step runs the flow
 * network (vio_initnet_*) on each keypoint to be tracked, between its
 * previous and current frame of the same camera, before tracking. A keypoint
 * whose proposal has confidence >= min_conf is tracked, with the
 * forward-backward check, over levels start_level..0 only, from p + flow; if
 * that track does not end VIO_TRACK_OK, or has not converged (max_last_step
 * > 0 and its last level-0 Gauss-Newton step moved the pattern by more than
 * max_last_step px: |dx| + |dy| + 7.62 |dtheta|), or the confidence is
 * lower, the keypoint is tracked exactly as without the network (whole
 * pyramid, start at p). A converged track sits at the optimum its start
 * leads to, so where the plain track converges too the two agree. Stereo
 * matching is unchanged. d_packed: the packed weights
 * (vio_initnet_pack, 16-byte aligned), read by every step and owned by the
 * caller, which keeps them alive while the initializer is on; NULL turns it
 * off. level_a and level_b must lie in 1 .. n_levels - 1 (upper levels),
 * start_level below n_levels; at most 128 streams (else
 * VIO_ERR_UNSUPPORTED). */
typedef struct {
  int32_t level_a, level_b;  /* pyramid levels of the network input          */
  int32_t start_level;       /* LK levels tracked from the proposal          */
  float min_conf;            /* confidence gate                              */
  float max_last_step;       /* convergence gate (px), <= 0: none            */
} vio_initnet_cfg;

vio_status vio_frontend_set_initnet(vio_frontend* fe, const void* d_packed,
                                    const vio_initnet_cfg* cfg);

/* --------------------------------------------------------------- batch -- */
/* Many stereo streams of mixed sizes in one step (the frontend of Sec. III-B
 * for each stream; batching streams is not in the paper). Streams are
 * grouped by size (up to 8 groups); every step runs the same three launches
 * for all groups (one per stage), optionally replayed from a captured CUDA
 * graph. Each stream keeps its own state on the device: its two frame
 * slots, keypoint lists, ids and first-frame flag; a step advances only the
 * streams marked active, the others keep their state untouched. */
typedef struct vio_batch vio_batch;

typedef struct {
  vio_params params;   /* per-group frontend parameters                   */
  int32_t w, h;        /* frame size; frames have pitch w                  */
  int32_t n_streams;   /* streams of this size                             */
  int32_t capacity;    /* keypoint slots per camera (gx*gy*k..32767)       */
} vio_stream_group;

/* Tunables of a batch step: threads per block of the tracking launches (32,
 * 64, 128, 256 or 512; one warp tracks one keypoint, so small blocks spread
 * the warps evenly over the SMs), the pyramid tile scale (-1, 0, 1: half, default, double
 * the deepest-level tile side), the order of stereo matching (0: every
 * cell's candidates are matched beside temporal tracking; 1: only the
 * selected keypoints are matched, after selection, in two more launches),
 * the pyramid levels the fused pyramid+detection launch computes (1..4,
 * 0 = up to 4; the rest follow in further pyramid launches: fewer levels per
 * pass recompute less of the halo of level 0), the CTA size of that launch
 * (128 or 256) and the warps that score one detection cell (1, 2, 4 or 8, at
 * most CTA size / 32; 0 = chosen from the launch: one when its cells fill the
 * GPU, more for few cells). Every setting gives the same lists bit for bit. */
typedef struct vio_batch_tune_s {
  int32_t k2_threads;
  int32_t pyr_tile_shift;
  int32_t stereo_after_select;
  int32_t pyr_first_levels;
  int32_t k1_threads;
  int32_t det_warps;
} vio_batch_tune;

vio_status vio_batch_create(vio_batch** out, const vio_stream_group* groups, int32_t n_groups);
/* Device bytes vio_batch_create would allocate for these groups (host only;
 * the same validation, the same errors). */
vio_status vio_batch_device_bytes(const vio_stream_group* groups, int32_t n_groups,
                                  int64_t* bytes);
vio_status vio_batch_destroy(vio_batch* b);

/* Device address of the frame (both cameras, 2 x h x w uint8, camera 1 at
 * + h*w) that stream `s` of group `g` reads at its next active step. Upload
 * the frame there (on the step's stream) before the step. The other slot
 * holds the stream's previous frame and must not be written. */
vio_status vio_batch_next_frame(vio_batch* b, int32_t g, int32_t s, uint8_t** d_frame);

/* One step of every stream whose entry of `active` (host array, one int32
 * per stream, groups in order) is nonzero; NULL = all streams. With graphs
 * enabled (vio_batch_set_graph) the launches are replayed from two captured
 * graphs; the first graph step captures them (make it outside any other
 * capture, on a stream other than the legacy default stream, else
 * VIO_ERR_INVALID_ARG). */
vio_status vio_batch_step(vio_batch* b, const int32_t* active, void* stream);
vio_status vio_batch_set_graph(vio_batch* b, int32_t enable);
vio_status vio_batch_set_tune(vio_batch* b, const vio_batch_tune* t);
vio_status vio_batch_get_tune(vio_batch* b, vio_batch_tune* t);

/* Times every tunable combination (180) over `reps` pairs of steps (a first frame,
 * then a tracked frame, all streams active) on the frames the caller has put
 * in BOTH slots of every stream, keeps the fastest, and resets every stream.
 * *best_ms: the chosen combination's time per tracked step. Blocking. */
vio_status vio_batch_autotune(vio_batch* b, int32_t reps, void* stream, float* best_ms);

/* Forget stream s of group g (its next step only detects). Enqueued. */
vio_status vio_batch_reset_stream(vio_batch* b, int32_t g, int32_t s, void* stream);

/* Output views of group g (layout as vio_frontend_view; the lists shown are
 * those of each stream's last step). Each stream's current list parity is
 * returned in parity[s] (host array of the group's n_streams, may be NULL);
 * the stream's lists are at slot base ((parity*n_streams + s)*2 + c) *
 * capacity of d_track_*, counts at (parity*n_streams + s)*2 + c. */
vio_status vio_batch_get_view(vio_batch* b, int32_t g, vio_frontend_view* out,
                              int32_t* parity);
int32_t vio_batch_launches_per_step(const vio_batch* b);

/* Per-step counters of group g (layout and meaning as vio_frontend_read_stats;
 * a stream's entry of a step in which it was inactive is all zero). Blocking.
 * *n_steps: the group's steps since create (the ring entry of step i is
 * i mod VIO_STATS_RING). */
vio_status vio_batch_read_stats(vio_batch* b, int32_t g, int32_t* host_out, int64_t* n_steps);

/* vio_frontend_set_initnet for every stream of the batch (one network and
 * configuration for all groups; every group needs the levels). Captured
 * graphs are re-captured at the next graph step. */
vio_status vio_batch_set_initnet(vio_batch* b, const void* d_packed, const vio_initnet_cfg* cfg);


/* ---------------------------------------------------------------- serving -- */
/* A request loop over a vio_batch (an addition; the paper runs one camera
 * rig per process). Size classes are vio_stream_group entries whose
 * n_streams is the number of concurrent sessions wanted; vio_server_plan
 * fits them into a device-memory budget (every class keeps at least one
 * slot; beyond that all classes scale down together) and vio_server_create
 * allocates exactly that. A session (one client stereo stream) is admitted
 * to a free slot of its class at open, or waits in the class's FIFO until a
 * session of that class closes; its pyramids, lists and frames stay on the
 * device while it holds the slot. Frames are uploaded as they arrive, from
 * PINNED host memory that the caller keeps until the frame's completion,
 * into per-slot staging buffers on an upload stream; whenever no step is on
 * the GPU, every admitted session with an uploaded frame joins the next
 * batch step (continuous batching), so uploads overlap the step in flight.
 * Each session's results are those of the same stream run alone through
 * vio_frontend. Host-side calls are not thread-safe: drive a server from one
 * thread. Times are seconds of vio_server_now()'s clock. */
typedef struct vio_server vio_server;

#define VIO_SERVER_LAST 1   /* submit flag: the session closes after this frame */

typedef struct {
  int64_t session;
  double t_offset;          /* arrival, seconds after the trace starts (ascending) */
  const uint8_t* host_frame;  /* pinned, 2 x h x w (camera 1 at + h*w)             */
  int64_t tag;
  int32_t flags;
} vio_server_req;

typedef struct {
  int64_t session, tag;
  double t_arrival, t_launch, t_done;  /* arrival, its step's launch, completion seen */
  int32_t n_tracks[2];                 /* list lengths of cameras 0 and 1 after it   */
  int32_t n_new;                       /* detections of this frame                   */
  int32_t status;                      /* VIO_OK, or the error of its step           */
} vio_server_done;

double vio_server_now(void);
/* Host only: slots per class (slots_out[n_classes]) and their device bytes
 * for a budget; VIO_ERR_OOM if even one slot per class does not fit. */
vio_status vio_server_plan(const vio_stream_group* classes, int32_t n_classes,
                           int64_t budget_bytes, int32_t* slots_out, int64_t* bytes_out);
vio_status vio_server_create(vio_server** out, const vio_stream_group* classes,
                             int32_t n_classes, int64_t budget_bytes);
vio_status vio_server_destroy(vio_server* s);
vio_status vio_server_slots(const vio_server* s, int32_t cls, int32_t* n_slots,
                            int64_t* device_bytes);
vio_status vio_server_set_initnet(vio_server* s, const void* d_packed,
                                  const vio_initnet_cfg* cfg);
vio_status vio_server_set_tune(vio_server* s, const vio_batch_tune* t);
/* New session of class cls; *admitted = 1 if it holds a slot now. */
vio_status vio_server_open(vio_server* s, int32_t cls, int64_t* session, int32_t* admitted);
/* Optional host buffers that receive the session's lists after each of its
 * frames: xy 2 x capacity float2, id 2 x capacity int32, count 2 int32. */
vio_status vio_server_set_output(vio_server* s, int64_t session, float* host_xy,
                                 int32_t* host_id, int32_t* host_count);
vio_status vio_server_submit(vio_server* s, int64_t session, const uint8_t* host_frame,
                             double t_arrival, int64_t tag, int32_t flags);
/* The session's queued frames still run; then its slot goes to the next
 * waiting session of its class. A waiting session leaves the queue. */
vio_status vio_server_close(vio_server* s, int64_t session);
/* Non-blocking progress: completes the step in flight if it has finished,
 * starts uploads, launches the next step if none is in flight. *n_done:
 * completions waiting to be taken. */
vio_status vio_server_poll(vio_server* s, int32_t* n_done);
int32_t vio_server_take(vio_server* s, vio_server_done* out, int32_t max);
/* Replays n requests in real time (submitting each at its offset, polling in
 * between) until all n have completed; out receives the n completions in
 * completion order. VIO_ERR_TIMEOUT after timeout_s seconds. */
vio_status vio_server_run_trace(vio_server* s, const vio_server_req* reqs, int64_t n,
                                vio_server_done* out, double timeout_s, int64_t* n_steps);
/* Host side of the last vio_server_run_trace: the longest time between two
 * passes of its loop (a loop that was not scheduled on a CPU delays every
 * request it holds) and the number of passes that took longer than 1 ms. */
vio_status vio_server_loop_stats(const vio_server* s, double* max_gap_s, int64_t* n_over_1ms);
/* Scheduling of vio_server_run_trace's host loop, for a loop that must not
 * lose its CPU (every request it holds waits while it does): pin_cpu >= 0
 * pins the calling thread to that CPU for the call, -2 to the CPU it is on
 * when the call starts, -1 leaves the affinity alone; rt_priority in 1..99
 * runs the call at that SCHED_FIFO priority, 0 leaves the policy alone. The
 * previous affinity and policy are restored when the call returns. Where the
 * system refuses (no permission), the loop runs unchanged:
 * vio_server_loop_policy_granted reports what the last trace got (bit 0:
 * pinned, bit 1: real-time). Default: -1, 0. */
vio_status vio_server_set_loop_policy(vio_server* s, int32_t pin_cpu, int32_t rt_priority);
vio_status vio_server_loop_policy_granted(const vio_server* s, int32_t* granted);

/* ---------------------------------------------------------------------------
 * Learned flow initializer. Not in the paper: its tracker starts each
 * keypoint from a position predicted through the camera model and the pose
 * (Sec. III-E); without that prediction, the starting point of a large motion
 * is where a plain zero start fails. This small network proposes the start:
 *
 *   input  4 x 16 x 16: source and target patch at pyramid levels a and b,
 *          16 x 16 integer grid from floor(p / 2^l + 0.5) - 8, value
 *          (v - 128) / 64, 0 outside the level;
 *   conv   3 x (3x3, stride 2, zero padding 1, 32 channels, ReLU),
 *          16 -> 8 -> 4 -> 2;
 *   fc     flatten (channel, row, column) 128 -> 64 + ReLU -> 3;
 *   output flow = 16 px * (o0, o1) (level-0 pixels), confidence = sigmoid(o2);
 *   loss   (o0 - fx/16)^2 + (o1 - fy/16)^2 + BCE(sigmoid(o2), y), y = 1 when
 *          the predicted flow is within the label radius r of the target (no
 *          gradient through y); the batch loss is the mean. The confidence
 *          thus estimates the chance that the proposal lies within r px; r
 *          is chosen to match the tracking start level's reach.
 *
 * Parameters: FP32 master vector of VIO_INITNET_N_PARAMS floats in the order
 * w1 (32,4,3,3), b1, w2 (32,32,3,3), b2, w3 (32,32,3,3), b3, w4 (64,128), b4,
 * w5 (3,64), b5 (row-major). Inference and the training forward pass run on
 * a packed copy (VIO_INITNET_PACKED_BYTES, 16-byte aligned): BF16 weights and
 * FP32 biases, written by vio_initnet_pack. Activations are BF16 between
 * layers, accumulation is FP32. Inputs x are BF16 bit patterns (uint16),
 * [n][4][16][16], 16-byte aligned. All calls are enqueued on `stream`;
 * pointers are device pointers owned by the caller.
 * ------------------------------------------------------------------------- */
#define VIO_INITNET_N_PARAMS 28131
#define VIO_INITNET_PACKED_BYTES 58016

vio_status vio_initnet_pack(const float* d_master, void* d_packed, void* stream);

/* Network inputs of n_images x capacity keypoints: image i's points at
 * d_pts[2*(i*capacity + k)] (level-0 x, y), its count at d_count[i] (NULL =
 * all capacity); `src` and `dst` are pyramids of one layout with n_images
 * each; point k of image i reads src image i and dst image i. Rows beyond
 * the count are zero. d_x: [n_images*capacity][4][16][16] bf16. */
vio_status vio_initnet_extract(const vio_pyr_layout* layout, const vio_pyr_batch* src,
                               const vio_pyr_batch* dst, const float* d_pts,
                               const int32_t* d_count, int32_t capacity, int32_t level_a,
                               int32_t level_b, uint16_t* d_x, void* stream);

/* d_out[3*i..3*i+2] = (dx, dy, confidence) of input i, i < n. Runs on the
 * tcgen05 tensor cores (BF16 operands, FP32 accumulation). */
vio_status vio_initnet_forward(const void* d_packed, const uint16_t* d_x, int32_t n,
                               float* d_out, void* stream);

/* Reads and clears (synchronously) the status word of the tensor-core
 * forward passes of this device (vio_initnet_forward and the learned
 * proposals of the frame steps): VIO_OK, or VIO_ERR_TIMEOUT when a launch
 * gave up waiting for an MMA completion (bounded polling), freed its tensor
 * memory and left its outputs unwritten. */
vio_status vio_initnet_fault(int32_t* status);

/* Adds grad_scale * (sum over the n samples d_index[0..n-1] (NULL = 0..n-1)
 * of dL_i/dparams), labels at radius label_radius px (> 0), to d_grad
 * (VIO_INITNET_N_PARAMS floats, gradient with respect to the master
 * parameters through the BF16 packing taken as the identity) and the sum of
 * the n losses to *d_loss. Targets: d_flow[2*j] =
 * (fx, fy) of sample j in level-0 pixels. The caller zeroes d_grad and
 * d_loss first. The forward pass is that of vio_initnet_forward. */
vio_status vio_initnet_train_step(const void* d_packed, const uint16_t* d_x,
                                  const float* d_flow, const int32_t* d_index, int32_t n,
                                  float grad_scale, float label_radius, float* d_grad,
                                  float* d_loss, void* stream);

/* Adam (Kingma and Ba, 2015) on the master parameters, step t >= 1:
 * m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2;
 * w -= lr (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps). */
vio_status vio_initnet_adam(float* d_master, const float* d_grad, float* d_m, float* d_v,
                            int32_t step, float lr, float beta1, float beta2, float eps,
                            void* stream);

#ifdef __cplusplus
}
#endif
#endif /* VIO_H_ */
