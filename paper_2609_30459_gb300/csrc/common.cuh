// Internal declarations shared by the libvio translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "vio.h"

namespace vio {

constexpr int kWarp = 32;
constexpr int kPatternMax = 64;   // 2 points per lane

// Pyramid geometry + batch as kernel parameters (passed by value).
struct Geom {
  int n_levels;
  int w[VIO_MAX_LEVELS], h[VIO_MAX_LEVELS], pitch[VIO_MAX_LEVELS];
  long long off[VIO_MAX_LEVELS];
};
struct Batch {
  const uint8_t* l0;
  long long l0_stride;
  uint8_t* upper;
  long long upper_stride;
  int n;
};

// Row/column split of a linear index without an integer division: for
// i < 2^22 the product (i + 0.5) * fl(1/w) is within (i/w) * 2^-23 of the
// exact quotient, less than the 0.5/w that separates it from the next
// integer, so its truncation is floor(i / w).
struct Split {
  float inv;
  int w;
  __device__ __forceinline__ explicit Split(int w_) : inv(1.f / (float)w_), w(w_) {}
  __device__ __forceinline__ void operator()(int i, int& r, int& c) const {
    r = (int)(((float)i + 0.5f) * inv);
    c = i - r * w;
  }
};

// SMs of the current device (cached per device; 152 if the query fails).
inline int sm_count() {
  static int n[32] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 32) return 152;
  if (n[dev] == 0) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v < 1)
      v = 152;
    n[dev] = v;
  }
  return n[dev];
}

// Host-side set-up that must run once on every device that launches a kernel
// (function attributes are per device): f() runs under a lock the first time
// a device is current here; its error is returned and the set-up is retried
// at the next call.
struct PerDeviceOnce {
  std::mutex mu;
  bool done[64] = {};
};
template <class F>
inline cudaError_t once_per_device(PerDeviceOnce& o, F f) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return f();
  std::lock_guard<std::mutex> lock(o.mu);
  if (o.done[dev]) return cudaSuccess;
  e = f();
  if (e == cudaSuccess) o.done[dev] = true;
  return e;
}

// The detection parameters of vio_params (cells, k, thresholds, border), as
// every detection entry point validates them.
inline bool detect_params_ok(const vio_params* p) {
  if (!p) return false;
  if (p->cell_w < 1 || p->cell_h < 1 || p->cell_w > 512 || p->cell_h > 512) return false;
  if (p->k_per_cell < 1 || p->k_per_cell > VIO_MAX_K) return false;
  if (p->n_thresholds < 1 || p->n_thresholds > VIO_MAX_THRESHOLDS) return false;
  for (int i = 0; i < p->n_thresholds; ++i) {
    if (p->thresholds[i] < 0 || p->thresholds[i] > 254) return false;
    // the sequence must not increase: the one-pass form relies on nesting
    if (i > 0 && p->thresholds[i] > p->thresholds[i - 1]) return false;
  }
  if (p->select_mode < VIO_SELECT_WARP_MAX || p->select_mode > VIO_SELECT_ATOMIC) return false;
  if (p->select_mode == VIO_SELECT_ATOMIC && p->k_per_cell != 1) return false;
  return p->detect_border >= 0;
}

inline Geom make_geom(const vio_pyr_layout& L) {
  Geom g{};
  g.n_levels = L.n_levels;
  for (int l = 0; l < VIO_MAX_LEVELS; ++l) {
    g.w[l] = L.w[l];
    g.h[l] = L.h[l];
    g.pitch[l] = L.pitch[l];
    g.off[l] = L.offset[l];
  }
  return g;
}
inline Batch make_batch(const vio_pyr_batch& b) {
  return Batch{b.d_level0, (long long)b.level0_stride, b.d_upper, (long long)b.upper_stride,
               b.n_images};
}

__device__ __forceinline__ const uint8_t* level_ptr(const Geom& g, const Batch& b, int img,
                                                    int l) {
  return l == 0 ? b.l0 + (long long)img * b.l0_stride
                : b.upper + (long long)img * b.upper_stride + g.off[l];
}
__device__ __forceinline__ uint8_t* level_ptr_mut(const Geom& g, const Batch& b, int img,
                                                  int l) {
  return b.upper + (long long)img * b.upper_stride + g.off[l];
}

// Track parameters shared by the tracking kernels.
struct TrackCfg {
  int gn_iters;
  int fb;
  float fb_max_dist;
  int top;            // first (coarsest) level tracked; -1 = n_levels - 1
};

__host__ __device__ inline int top_level(const TrackCfg& c, const Geom& g) {
  return c.top < 0 ? g.n_levels - 1 : c.top;
}

}  // namespace vio

// The context: parameters plus scratch sized at creation.
struct vio_ctx {
  vio_params p;
  int max_w, max_h, max_images;
  int max_cells;
  // detection scratch: per image, per cell, k packed candidate keys + count
  unsigned long long* d_cand;
  int32_t* d_cand_count;
  // device status word (VIO_OK, or the first device-side error, e.g. a
  // bounded wait that gave up) and its pinned host copy
  int32_t* d_status;
  int32_t* h_status;
};

namespace vio {
// launchers (host side), implemented in the .cu files
cudaError_t launch_pyramid(const Geom& g, const Batch& b, int round_mode, cudaStream_t s);
cudaError_t launch_pyramid_from(const Geom& g, const Batch& b, int s0, int round_mode,
                                cudaStream_t s);
cudaError_t launch_fast_scores(const uint8_t* img, int w, int h, int pitch, int16_t* out,
                               cudaStream_t s);
cudaError_t launch_detect(const vio_params& p, const Geom& g, const Batch& b,
                          const uint8_t* occ, const uint8_t* mask, long long mask_stride,
                          unsigned long long* cand, int32_t* cand_count, float* kp,
                          int16_t* score, int32_t* count, int capacity, cudaStream_t s);
cudaError_t launch_select(const unsigned long long* cand, const int32_t* cand_count,
                          const uint8_t* occ, int n_cells, int k, int w, float* kp,
                          int16_t* score, int32_t* count, int capacity, int n_images,
                          cudaStream_t s);
cudaError_t launch_track(const Geom& g, const Batch& src, const Batch& dst, const float* pts,
                         const float* init, const int32_t* count, int capacity,
                         const TrackCfg& cfg, float* out3, float* out2, uint8_t* status,
                         float* fb_dist, cudaStream_t s, bool shared_pts = false,
                         float* last_step = nullptr);
cudaError_t launch_fb_check(const float* orig, const float* back, const int32_t* count,
                            int capacity, int n_images, float max_dist, uint8_t* status,
                            float* dist, cudaStream_t s);
}  // namespace vio
