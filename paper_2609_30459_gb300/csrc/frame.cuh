// Launch description of one frontend frame (frame.cu), for one or more
// groups of same-size stereo streams merged into the same three launches.
#pragma once
#include "common.cuh"

namespace vio {

constexpr int kMaxGroups = 8;

// Launch tunables (chosen by the autotuner of a batch).
struct FrameTune {
  int k2_threads;      // threads per block of the tracking launch (64..512)
  int pyr_tile_shift;  // deepest-level pyramid tile side = (32 >> (m-1)) << shift
  int stereo_after;    // 1: stereo-match only the selected keypoints, after selection
  int pyr_first;       // pyramid levels of K1's fused pass (1..4; 0 = as many as fit)
  int k1_threads;      // CTA size of K1: 128 or 256
  int det_warps;       // warps per detection cell (1, 2, 4, 8; 0 = from the launch size)
};

struct FrameLaunch {
  vio_params p;
  Geom g;
  int n_streams, cap;
  // Images. Unslotted: stream s camera c is image 2s+c of `cur` (this frame)
  // and of `prev` (previous frame). Slotted: `cur` == `prev` holds two frame
  // slots per stream and stream s at parity q uses image 2(q*ns + s) + c,
  // the previous frame being at parity 1 - q.
  Batch cur, prev;
  int slotted;
  int host_parity, host_have_prev;  // unslotted: list parity and first-frame flag
  int32_t* parity;                  // slotted, per stream (flipped by finalize)
  int32_t* have_prev;               // slotted, per stream
  const int32_t* active;            // slotted, per stream, nonzero = step it (null: all)
  // keypoint lists [parity][stream][camera] x cap
  float* list_xy;
  int32_t* list_id;
  int32_t* list_count;
  uint8_t* list_status;
  // temporal results [stream][camera] x cap
  float* trk_xy;
  uint8_t* trk_status;
  unsigned long long* cand;        // candidates, ns x cells x k
  int32_t* cand_count;             // ns x cells
  float* spec_xy;                  // stereo results of the candidates, ns x cells x k
  uint8_t* spec_status;
  float* new_xy;                   // ns x cap
  int32_t* new_count;              // ns
  int32_t* next_id;                // ns
  uint8_t* occupancy;              // ns x cells
  int32_t* stats;                  // ring, VIO_STATS_RING x ns x VIO_N_STATS
  int32_t* step_ctr;               // incremented once per launch of the frame
  int32_t* ctr_copy;               // nullable: K1 also stores the new count here and the
                                   // later launches of the step read it from here (so the
                                   // next step's K1 may run beside them)
  // learned flow initializer of temporal tracking (net == null: off)
  const void* net;                 // packed weights
  int net_la, net_lb, net_top;
  float net_tau;
  float net_max_step;   // convergence gate of a learned track (<= 0: none)
  float* net_out;                  // [stream][camera] x cap x (dx, dy, conf)
  uint8_t* trk_learned;            // [stream][camera] x cap: 1 = tracked from the proposal
  int stereo_after;                // set by launch_frames from the tune
};

// Per-stream view of a FrameLaunch.
struct StreamRef {
  int cur_img, prev_img;   // image index of camera 0
  int li, lo;              // list parity in / out
  bool have_prev, active;
};

__host__ __device__ inline StreamRef stream_ref(const FrameLaunch& f, int s) {
  StreamRef r;
  if (!f.slotted) {
    r.cur_img = 2 * s;
    r.prev_img = 2 * s;
    r.li = f.host_parity;
    r.lo = f.host_parity ^ 1;
    r.have_prev = f.host_have_prev != 0;
    r.active = true;
    return r;
  }
#ifdef __CUDA_ARCH__
  const int q = f.parity[s];
  r.cur_img = 2 * (q * f.n_streams + s);
  r.prev_img = 2 * ((q ^ 1) * f.n_streams + s);
  r.li = q;
  r.lo = q ^ 1;
  r.have_prev = f.have_prev[s] != 0;
  r.active = f.active ? f.active[s] != 0 : true;
#else
  r = StreamRef{};
#endif
  return r;
}

// Enqueues one frame of every group on `s` (3 launches, plus one pyramid
// pass per group for levels beyond 5, plus the flow proposals when the
// groups' initializer is on). marks: VIO_N_STAGES + 1 events recorded at the
// stage boundaries (or null).
// part: 0 the whole step; 1 only its front (pyramids and detection
// candidates: K1 and the deeper pyramid levels); 2 the rest. The front of a
// step reads only its own frames and writes the current pyramid ring slot and
// the candidate buffers, so it may run beside the rest of the previous step
// when those are not the previous step's.
cudaError_t launch_frames(const FrameLaunch* f, int n_groups, const FrameTune& tune,
                          cudaStream_t s, cudaEvent_t* marks, int part = 0);
int frame_launches(const Geom* g, int n_groups, bool with_net, bool stereo_after,
                   int pyr_first);

// Keypoint lists (2 per stream) one launch of the proposal kernel handles.
constexpr int KN_MAX_LISTS = 256;

// Initializer configuration check: input levels in 1 .. n_levels - 1, start
// level below n_levels, a finite gate, 16-byte aligned weights.
inline bool initnet_cfg_ok(const vio_initnet_cfg* c, int n_levels, const void* packed) {
  if (!c || ((uintptr_t)packed & 15)) return false;
  // the network reads upper pyramid levels only (aligned rows)
  if (c->level_a < 1 || c->level_b < 1 || c->start_level < 0) return false;
  if (c->level_a >= n_levels || c->level_b >= n_levels || c->start_level >= n_levels)
    return false;
  return c->min_conf == c->min_conf && c->max_last_step == c->max_last_step;   // not NaN
}
int frame_front_smem(const Geom& g, const vio_params& p, int tile_shift, int pyr_first,
                     int threads, int det_warps);

}  // namespace vio
