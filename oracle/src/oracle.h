/*
 * CPU oracle of the VkVIO stereo frontend (arxiv 2609.30459, Sec. III).
 *
 * TEST INFRASTRUCTURE ONLY. This code exists to check the CUDA path; the
 * product never links, loads or calls it. Only the tests, the smoke check and
 * the CPU-baseline leg of the benchmark use it. It shares no code, header or
 * table with the CUDA library: every definition below is restated here from
 * the paper on its own.
 *
 * Precision: integer arithmetic where the paper fixes it (pyramid, FAST,
 * selection), FP64 everywhere else (tracking).
 *
 * Each function is plain and slow on purpose: no blocking, fusion or
 * reordering beyond what the cited passage states.
 */
#pragma once
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Per-keypoint track status (the oracle's own numbering, identical by value to
 * the library's so that tests can compare arrays directly). */
enum {
  VO_OK = 0,
  VO_OOB_TEMPLATE = 1, /* template samples leave the image at level 0 */
  VO_OOB_WARP = 2,     /* a warped sample leaves the target image */
  VO_DEGENERATE_H = 3, /* Gauss-Newton Hessian not positive definite */
  VO_ZERO_MEAN = 4,    /* patch mean <= 0: Eq. 4 undefined */
  VO_FB_FAIL = 5,      /* forward-backward distance above the threshold */
  VO_NAN = 6           /* non-finite increment */
};

/* One image plane: uint8, row-major, `pitch` bytes between rows. */
typedef struct {
  const uint8_t* data;
  int32_t w, h, pitch;
} vo_image;

#define VO_MAX_LEVELS 8
typedef struct {
  vo_image lv[VO_MAX_LEVELS];
  int32_t n_levels;
} vo_pyramid;

/* ---- Sec. III-C, Eq. 1: one pyramid level from the previous one. ----------
 * dst is floor(w/2) x floor(h/2). round_mode 0 = nearest (half up), 1 = floor
 * (the ">> 8" of Eq. 3). Border: clamp to edge. */
void vo_pyr_down(const uint8_t* src, int32_t w, int32_t h, int32_t src_pitch,
                 uint8_t* dst, int32_t dst_pitch, int32_t round_mode);

/* ---- Sec. III-D: FAST-9 score of every pixel. -----------------------------
 * score = largest integer tau >= 0 such that 9 contiguous pixels of the
 * 16-pixel radius-3 Bresenham ring are all brighter than I(p)+tau or all
 * darker than I(p)-tau; -1 if no tau >= 0 qualifies or the ring leaves the
 * image (valid region 3 <= x <= w-4, 3 <= y <= h-4). */
void vo_fast_scores(const uint8_t* img, int32_t w, int32_t h, int32_t pitch,
                    int16_t* score /* w*h, row-major, pitch w */);

/* FAST ring offsets in order (exported so tests can check the geometry). */
void vo_fast_ring(int32_t* dx /*16*/, int32_t* dy /*16*/);

/* ---- Sec. III-D: grid-cell detection. ------------------------------------ */
typedef struct {
  int32_t cell_w, cell_h;      /* cell size in level-0 pixels              */
  int32_t k;                   /* per-cell keypoint limit                  */
  int32_t n_thresholds;        /* length of the threshold sequence         */
  int32_t thresholds[8];       /* descending, e.g. 40,20,10,5              */
  int32_t border;              /* candidates need border<=x<=w-1-border    */
} vo_detect_params;

/* Detection on one image. occupancy: per-cell count of existing tracks
 * (uint8, grid raster order, may be NULL); mask: per-pixel, 0 = excluded (may
 * be NULL). Writes at most `capacity` keypoints in cell raster order, then by
 * rank; returns the number written. one_pass = 0 runs the threshold sequence
 * literally, 1 takes the top k of all candidates at the smallest threshold. */
int32_t vo_detect_grid(const uint8_t* img, int32_t w, int32_t h, int32_t pitch,
                       const vo_detect_params* p, const uint8_t* occupancy,
                       const uint8_t* mask, int32_t mask_pitch,
                       float* kp_xy /* capacity*2 */, int16_t* kp_score,
                       int32_t capacity, int32_t one_pass);

/* ---- Sec. III-E: patch tracking. ----------------------------------------- */
typedef struct {
  int32_t gn_iters;       /* Gauss-Newton iterations per level (5)          */
  int32_t pattern_id;     /* 0 = the 52-point odd lattice                   */
  double fb_max_dist;     /* forward-backward threshold, level-0 px         */
} vo_track_params;

/* Number of points and offsets of a sample pattern. */
int32_t vo_pattern(int32_t pattern_id, double* u, double* v /* >= 64 each */);

/* Track n keypoints from src to dst, coarse to fine over the levels both
 * pyramids share. pts: n*(x,y) in level-0 px (float32, as the library gets
 * them). init: n*(tx,ty,theta) or NULL for the identity (t = p, theta = 0).
 * fb = 1 runs the backward pass and the distance check.
 * Outputs: warp n*(tx,ty,theta) in level-0 px (forward result), status n,
 * fb_dist n (NaN where not computed), margin n (smallest distance, in level-0
 * px, between any bound test's value and its bound; used to explain status
 * disagreements), back n*(tx,ty,theta) (backward result, may be NULL),
 * last_step n (how far the forward pass's last level-0 Gauss-Newton step
 * moved the pattern: |dx| + |dy| + r |dtheta|, r the pattern's radius; NaN if
 * the forward pass failed; may be NULL). */
void vo_track(const vo_pyramid* src, const vo_pyramid* dst, int32_t n,
              const float* pts, const float* init, const vo_track_params* p,
              int32_t fb, double* warp, uint8_t* status, double* fb_dist,
              double* margin, double* back, double* last_step, int32_t n_threads);

/* Template quantities at one level, for the tests (Sec. III-E): samples s,
 * gradients gx, gy, Jacobian rows J (np*3), Hessian H (9) and gain G (3*np),
 * all of the mean-normalised patch. Returns a status (VO_OK or the failure). */
int32_t vo_template(const vo_image* img, double qx, double qy,
                    int32_t pattern_id, double* s, double* gx, double* gy,
                    double* J, double* H, double* G, double* mean);

/* SE(2) exponential as used by Eq. 5: exp(dx,dy,dth) -> (R, t) as a 3x3
 * homogeneous matrix, row-major. */
void vo_se2_exp(double dx, double dy, double dth, double* M /* 9 */);

#ifdef __cplusplus
}
#endif
