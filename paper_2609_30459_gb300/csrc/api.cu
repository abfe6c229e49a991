// C ABI of libvio: parameters, pyramid layout, context, and the validated
// entry points of each stage. Every function checks its arguments before it
// enqueues anything.
#include <new>

#include "common.cuh"
#include "detect_dev.cuh"
#include "frame.cuh"
#include "pyramid_dev.cuh"

namespace {

bool params_ok(const vio_params* p) {
  if (!vio::detect_params_ok(p)) return false;
  if (p->n_levels < 1 || p->n_levels > VIO_MAX_LEVELS) return false;
  if (p->round_mode != 0 && p->round_mode != 1) return false;
  if (p->gn_iters < 0 || p->gn_iters > 1000) return false;
  if (p->pattern_id != 0) return false;
  if (!(p->fb_max_dist >= 0.f)) return false;
  return true;
}

bool layout_ok(const vio_pyr_layout* L) {
  if (!L || L->n_levels < 1 || L->n_levels > VIO_MAX_LEVELS) return false;
  for (int l = 0; l < L->n_levels; ++l)
    if (L->w[l] < 1 || L->h[l] < 1 || L->pitch[l] < L->w[l]) return false;
  for (int l = 1; l < L->n_levels; ++l) {
    if (L->w[l] != L->w[l - 1] / 2 || L->h[l] != L->h[l - 1] / 2) return false;
    if (L->offset[l] < 0 || L->offset[l] + (int64_t)L->pitch[l] * L->h[l] > L->upper_bytes)
      return false;
  }
  return true;
}

bool batch_ok(const vio_pyr_layout* L, const vio_pyr_batch* b) {
  if (!b || b->n_images < 1 || !b->d_level0) return false;
  if (b->n_images > 1 && b->level0_stride < (int64_t)L->pitch[0] * L->h[0]) return false;
  if (L->n_levels > 1) {
    if (!b->d_upper) return false;
    if (b->n_images > 1 && b->upper_stride < L->upper_bytes) return false;
    if (b->upper_stride % 16 != 0) return false;
  }
  return true;
}

vio_status cuda_status(cudaError_t e) { return e == cudaSuccess ? VIO_OK : VIO_ERR_CUDA; }

}  // namespace

extern "C" void vio_params_default(vio_params* p) {
  if (!p) return;
  *p = vio_params{};
  p->n_levels = 4;
  p->round_mode = 0;
  p->gn_iters = 5;
  p->pattern_id = 0;
  p->cell_w = 50;
  p->cell_h = 50;
  p->k_per_cell = 1;
  p->n_thresholds = 4;
  p->thresholds[0] = 40;
  p->thresholds[1] = 20;
  p->thresholds[2] = 10;
  p->thresholds[3] = 5;
  p->detect_border = 9;
  p->fb_max_dist = 0.2f;
}

extern "C" const char* vio_status_string(vio_status s) {
  switch (s) {
    case VIO_OK: return "ok";
    case VIO_ERR_INVALID_ARG: return "invalid argument";
    case VIO_ERR_CUDA: return "CUDA runtime error";
    case VIO_ERR_OOM: return "out of device memory";
    case VIO_ERR_TIMEOUT: return "device-side wait timed out";
    case VIO_ERR_UNSUPPORTED: return "unsupported";
    default: return "unknown status";
  }
}

extern "C" vio_status vio_pyr_layout_make(int32_t w, int32_t h, int32_t n_levels,
                                          int32_t level0_pitch, vio_pyr_layout* out) {
  if (!out || w < 1 || h < 1 || n_levels < 1 || n_levels > VIO_MAX_LEVELS || level0_pitch < w)
    return VIO_ERR_INVALID_ARG;
  vio_pyr_layout L{};
  L.n_levels = n_levels;
  L.w[0] = w;
  L.h[0] = h;
  L.pitch[0] = level0_pitch;
  int64_t off = 0;
  for (int l = 1; l < n_levels; ++l) {
    L.w[l] = L.w[l - 1] / 2;
    L.h[l] = L.h[l - 1] / 2;
    if (L.w[l] < 1 || L.h[l] < 1) return VIO_ERR_INVALID_ARG;
    L.pitch[l] = (L.w[l] + 127) & ~127;
    L.offset[l] = off;
    off += ((int64_t)L.pitch[l] * L.h[l] + 255) & ~(int64_t)255;
  }
  L.upper_bytes = off;
  *out = L;
  return VIO_OK;
}

extern "C" vio_status vio_ctx_create(vio_ctx** out, const vio_params* p, int32_t max_w,
                                     int32_t max_h, int32_t max_images) {
  if (!out || !params_ok(p) || max_w < 1 || max_h < 1 || max_images < 1)
    return VIO_ERR_INVALID_ARG;
  if (!vio::det::detect_fits(p->cell_w, p->cell_h, p->k_per_cell))
    return VIO_ERR_UNSUPPORTED;
  *out = nullptr;
  vio_ctx* c = new (std::nothrow) vio_ctx();
  if (!c) return VIO_ERR_OOM;
  c->p = *p;
  c->max_w = max_w;
  c->max_h = max_h;
  c->max_images = max_images;
  c->max_cells = (max_w / p->cell_w) * (max_h / p->cell_h);
  const size_t n = (size_t)c->max_images * (size_t)(c->max_cells > 0 ? c->max_cells : 1);
  if (cudaMalloc(&c->d_cand, n * p->k_per_cell * sizeof(unsigned long long)) != cudaSuccess ||
      cudaMalloc(&c->d_cand_count, n * sizeof(int32_t)) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(c->d_cand);
    delete c;
    return VIO_ERR_OOM;
  }
  *out = c;
  return VIO_OK;
}

extern "C" vio_status vio_ctx_destroy(vio_ctx* c) {
  if (!c) return VIO_ERR_INVALID_ARG;
  cudaFree(c->d_cand);
  cudaFree(c->d_cand_count);
  delete c;
  return VIO_OK;
}

extern "C" vio_status vio_pyramid_build(vio_ctx* ctx, const vio_pyr_layout* layout,
                                        const vio_pyr_batch* batch, void* stream) {
  if (!ctx || !layout_ok(layout) || !batch_ok(layout, batch)) return VIO_ERR_INVALID_ARG;
  if (layout->n_levels != ctx->p.n_levels) return VIO_ERR_INVALID_ARG;
  if (batch->n_images > 65535) return VIO_ERR_UNSUPPORTED;
  return cuda_status(vio::launch_pyramid(vio::make_geom(*layout), vio::make_batch(*batch),
                                         ctx->p.round_mode, (cudaStream_t)stream));
}

extern "C" vio_status vio_fast_scores(const uint8_t* d_img, int32_t w, int32_t h, int32_t pitch,
                                      int16_t* d_score, void* stream) {
  if (!d_img || !d_score || w < 1 || h < 1 || pitch < w || h > 65535 * 8)
    return VIO_ERR_INVALID_ARG;
  return cuda_status(vio::launch_fast_scores(d_img, w, h, pitch, d_score, (cudaStream_t)stream));
}

extern "C" vio_status vio_detect_grid(vio_ctx* ctx, const vio_pyr_layout* layout,
                                      const vio_pyr_batch* batch, const uint8_t* d_occupancy,
                                      const uint8_t* d_mask, int64_t mask_stride, float* d_kp,
                                      int16_t* d_score, int32_t* d_count, int32_t capacity,
                                      void* stream) {
  if (!ctx || !layout_ok(layout) || !d_kp || !d_score || !d_count || capacity < 0)
    return VIO_ERR_INVALID_ARG;
  if (!batch || batch->n_images < 1 || !batch->d_level0) return VIO_ERR_INVALID_ARG;
  if (batch->n_images > 1 && batch->level0_stride < (int64_t)layout->pitch[0] * layout->h[0])
    return VIO_ERR_INVALID_ARG;
  if (d_mask && batch->n_images > 1 && mask_stride < (int64_t)layout->w[0] * layout->h[0])
    return VIO_ERR_INVALID_ARG;
  if (layout->w[0] > ctx->max_w || layout->h[0] > ctx->max_h ||
      batch->n_images > ctx->max_images)
    return VIO_ERR_INVALID_ARG;
  if (batch->n_images > 65535) return VIO_ERR_UNSUPPORTED;
  return cuda_status(vio::launch_detect(ctx->p, vio::make_geom(*layout),
                                        vio::make_batch(*batch), d_occupancy, d_mask,
                                        mask_stride, ctx->d_cand, ctx->d_cand_count, d_kp,
                                        d_score, d_count, capacity, (cudaStream_t)stream));
}

extern "C" vio_status vio_pyramid_detect(vio_ctx* ctx, const vio_pyr_layout* layout,
                                         const vio_pyr_batch* batch, const uint8_t* d_occupancy,
                                         const uint8_t* d_mask, int64_t mask_stride,
                                         float* d_kp, int16_t* d_score, int32_t* d_count,
                                         int32_t capacity, void* stream) {
  if (!ctx || !layout_ok(layout) || !batch_ok(layout, batch) || !d_kp || !d_score ||
      !d_count || capacity < 0)
    return VIO_ERR_INVALID_ARG;
  if (layout->n_levels != ctx->p.n_levels) return VIO_ERR_INVALID_ARG;
  if (d_mask && batch->n_images > 1 && mask_stride < (int64_t)layout->w[0] * layout->h[0])
    return VIO_ERR_INVALID_ARG;
  if (layout->w[0] > ctx->max_w || layout->h[0] > ctx->max_h ||
      batch->n_images > ctx->max_images)
    return VIO_ERR_INVALID_ARG;
  if (batch->n_images > 65535) return VIO_ERR_UNSUPPORTED;
  const vio::Geom g = vio::make_geom(*layout);
  const vio::Batch b = vio::make_batch(*batch);
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = vio::launch_front(ctx->p, g, b, 1, d_mask, mask_stride, ctx->d_cand,
                                    ctx->d_cand_count, s);   // all levels
  if (e == cudaSuccess) {
    const int n_cells = (layout->w[0] / ctx->p.cell_w) * (layout->h[0] / ctx->p.cell_h);
    e = vio::launch_select(ctx->d_cand, ctx->d_cand_count, d_occupancy, n_cells,
                           ctx->p.k_per_cell, layout->w[0], d_kp, d_score, d_count, capacity,
                           batch->n_images, s);
  }
  return cuda_status(e);
}

extern "C" vio_status vio_track_patches(vio_ctx* ctx, const vio_pyr_layout* layout,
                                        const vio_pyr_batch* src, const vio_pyr_batch* dst,
                                        const float* d_pts, const float* d_init,
                                        const int32_t* d_count, int32_t capacity, int32_t flags,
                                        float* d_out, uint8_t* d_status, float* d_fb_dist,
                                        void* stream) {
  if (!ctx || !layout_ok(layout) || !batch_ok(layout, src) || !batch_ok(layout, dst))
    return VIO_ERR_INVALID_ARG;
  if (src->n_images != dst->n_images || !d_pts || !d_out || !d_status || capacity < 0)
    return VIO_ERR_INVALID_ARG;
  const int mode = flags & 0xf, from = (flags >> 4) & 0xf;
  if ((mode != VIO_TRACK_FORWARD && mode != VIO_TRACK_WITH_FB) || (flags & ~0xff) ||
      from > layout->n_levels)
    return VIO_ERR_INVALID_ARG;
  vio::TrackCfg cfg{ctx->p.gn_iters, mode == VIO_TRACK_WITH_FB ? 1 : 0, ctx->p.fb_max_dist,
                    from - 1};
  return cuda_status(vio::launch_track(vio::make_geom(*layout), vio::make_batch(*src),
                                       vio::make_batch(*dst), d_pts, d_init, d_count, capacity,
                                       cfg, d_out, nullptr, d_status, d_fb_dist,
                                       (cudaStream_t)stream));
}

extern "C" vio_status vio_stereo_match(vio_ctx* ctx, const vio_pyr_layout* layout,
                                       const vio_pyr_batch* cam0, const vio_pyr_batch* cam1,
                                       const float* d_pts, const float* d_init,
                                       const int32_t* d_count, int32_t capacity, float* d_match,
                                       uint8_t* d_status, float* d_fb_dist, void* stream) {
  if (!ctx || !layout_ok(layout) || !batch_ok(layout, cam0) || !batch_ok(layout, cam1))
    return VIO_ERR_INVALID_ARG;
  if (cam0->n_images != cam1->n_images || !d_pts || !d_match || !d_status || capacity < 0)
    return VIO_ERR_INVALID_ARG;
  vio::TrackCfg cfg{ctx->p.gn_iters, 1, ctx->p.fb_max_dist, -1};
  return cuda_status(vio::launch_track(vio::make_geom(*layout), vio::make_batch(*cam0),
                                       vio::make_batch(*cam1), d_pts, d_init, d_count, capacity,
                                       cfg, nullptr, d_match, d_status, d_fb_dist,
                                       (cudaStream_t)stream));
}

extern "C" vio_status vio_fb_check(const float* d_orig, const float* d_back,
                                   const int32_t* d_count, int32_t capacity, int32_t n_images,
                                   float max_dist, uint8_t* d_status, float* d_dist,
                                   void* stream) {
  if (!d_orig || !d_back || !d_status || capacity < 0 || n_images < 0 || !(max_dist >= 0.f))
    return VIO_ERR_INVALID_ARG;
  return cuda_status(vio::launch_fb_check(d_orig, d_back, d_count, capacity, n_images, max_dist,
                                          d_status, d_dist, (cudaStream_t)stream));
}
