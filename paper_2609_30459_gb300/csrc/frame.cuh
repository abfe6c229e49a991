// Launch description of one frontend frame (frame.cu).
#pragma once
#include "common.cuh"

namespace vio {

struct FrameLaunch {
  vio_params p;
  Geom g;
  int n_streams, cap, have_prev;
  Batch prev, cur;                 // previous / current frame: 2 images per stream
  const float* list_xy_in;         // lists of the previous step, (2*ns) x cap
  const int32_t* list_id_in;
  const int32_t* list_count_in;
  float* list_xy_out;              // lists after this step
  int32_t* list_id_out;
  int32_t* list_count_out;
  uint8_t* list_status;
  float* trk_xy;                   // temporal results, (2*ns) x cap
  uint8_t* trk_status;
  unsigned long long* cand;        // candidates, ns x cells x k
  int32_t* cand_count;             // ns x cells
  float* spec_xy;                  // stereo results of the candidates, ns x cells x k
  uint8_t* spec_status;
  float* new_xy;                   // ns x cap
  int32_t* new_count;              // ns
  int32_t* next_id;                // ns
  uint8_t* occupancy;              // ns x cells
  int32_t* stats;                  // ns x VIO_N_STATS
};

// Enqueues the frame on `s`. marks: 5 events recorded at the stage
// boundaries (or null).
cudaError_t launch_frame(const FrameLaunch& f, cudaStream_t s, cudaEvent_t* marks);
int frame_launches(const Geom& g);
// Fused pyramid (levels 1-4) and per-cell detection candidates of every
// det_step-th image of `all`, one launch.
cudaError_t launch_front(const vio_params& p, const Geom& g, const Batch& all, int det_step,
                         const uint8_t* mask, long long mask_stride, unsigned long long* cand,
                         int32_t* cand_count, cudaStream_t s);
int frame_front_smem(const Geom& g, const vio_params& p);

}  // namespace vio
