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
      cudaMalloc(&c->d_cand_count, n * sizeof(int32_t)) != cudaSuccess ||
      cudaMalloc(&c->d_status, sizeof(int32_t)) != cudaSuccess ||
      cudaMallocHost(&c->h_status, sizeof(int32_t)) != cudaSuccess ||
      cudaMemset(c->d_status, 0, sizeof(int32_t)) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(c->d_cand);
    cudaFree(c->d_cand_count);
    cudaFree(c->d_status);
    cudaFreeHost(c->h_status);
    delete c;
    return VIO_ERR_OOM;
  }
  *c->h_status = 0;
  *out = c;
  return VIO_OK;
}

extern "C" vio_status vio_ctx_destroy(vio_ctx* c) {
  if (!c) return VIO_ERR_INVALID_ARG;
  cudaFree(c->d_cand);
  cudaFree(c->d_cand_count);
  cudaFree(c->d_status);
  cudaFreeHost(c->h_status);
  delete c;
  return VIO_OK;
}

namespace {

// Polls *flag until it equals `value`, for at most timeout_ns of the GPU's
// global timer, and in any case at most max_polls polls (each a global load, a
// timer read and a short sleep); on giving up it records VIO_ERR_TIMEOUT in
// the status word (the first error recorded stays) and returns, so the
// context stays usable.
__global__ void wait_flag_kernel(const volatile int32_t* flag, int32_t value, long long timeout_ns,
                                 long long max_polls, int32_t* status) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  unsigned long long t0, t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
  for (long long i = 0; i < max_polls; ++i) {
    if (*flag == value) return;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    if ((long long)(t - t0) > timeout_ns) break;
    __nanosleep(1000);
  }
  if (*flag == value) return;
  atomicCAS(status, (int32_t)VIO_OK, (int32_t)VIO_ERR_TIMEOUT);
}

}  // namespace

extern "C" vio_status vio_wait_flag(vio_ctx* ctx, const int32_t* d_flag, int32_t value,
                                    int64_t timeout_ns, void* stream) {
  if (!ctx || !d_flag || timeout_ns < 0 || timeout_ns > 2000000000LL) return VIO_ERR_INVALID_ARG;
  // a poll (a global load and a timer read) takes well over 100 ns, so the
  // timer ends the wait first; the count only bounds it if the timer did not
  const long long max_polls = timeout_ns / 100 + 1024;
  wait_flag_kernel<<<1, 32, 0, (cudaStream_t)stream>>>(d_flag, value, timeout_ns, max_polls,
                                                       ctx->d_status);
  return cudaGetLastError() == cudaSuccess ? VIO_OK : VIO_ERR_CUDA;
}

extern "C" vio_status vio_ctx_sync(vio_ctx* ctx, void* stream, vio_status* device_status) {
  if (!ctx || !device_status) return VIO_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaMemcpyAsync(ctx->h_status, ctx->d_status, sizeof(int32_t), cudaMemcpyDeviceToHost,
                      s) != cudaSuccess ||
      cudaMemsetAsync(ctx->d_status, 0, sizeof(int32_t), s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return VIO_ERR_CUDA;
  *device_status = *ctx->h_status;
  return VIO_OK;
}

extern "C" vio_status vio_last_error(vio_ctx* ctx) {
  if (!ctx) return VIO_ERR_INVALID_ARG;
  int32_t v = 0;
  if (cudaMemcpy(&v, ctx->d_status, sizeof(int32_t), cudaMemcpyDeviceToHost) != cudaSuccess)
    return VIO_ERR_CUDA;
  return v;
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
  // Per chunk of images, the pyramid launch and then the detection launch:
  // each kernel runs at its own shape and occupancy (the single fused launch
  // of the per-frame step, kept there for its latency, runs both parts at the
  // larger one's), and a chunk's level 0 (at most 64 MiB, half the L2) is
  // still in L2 when the detection reads it, so DRAM serves it once.
  const int n_cells = (layout->w[0] / ctx->p.cell_w) * (layout->h[0] / ctx->p.cell_h);
  const long long img_bytes = (long long)layout->pitch[0] * layout->h[0];
  const long long by_l2 = (64LL << 20) / (img_bytes > 0 ? img_bytes : 1);
  const int chunk = (int)(by_l2 < 1 ? 1 : (by_l2 < b.n ? by_l2 : b.n));
  cudaError_t e = cudaSuccess;
  for (int i0 = 0; i0 < b.n && e == cudaSuccess; i0 += chunk) {
    vio::Batch bc = b;
    bc.l0 = b.l0 + (long long)i0 * b.l0_stride;
    bc.upper = b.upper + (long long)i0 * b.upper_stride;
    bc.n = b.n - i0 < chunk ? b.n - i0 : chunk;
    e = vio::launch_pyramid(g, bc, ctx->p.round_mode, s);
    if (e != cudaSuccess) break;
    e = vio::launch_detect(
        ctx->p, g, bc, d_occupancy ? d_occupancy + (long long)i0 * n_cells : nullptr,
        d_mask ? d_mask + (long long)i0 * mask_stride : nullptr, mask_stride,
        ctx->d_cand + (long long)i0 * n_cells * ctx->p.k_per_cell,
        ctx->d_cand_count + (long long)i0 * n_cells, d_kp + 2LL * i0 * capacity,
        d_score + (long long)i0 * capacity, d_count + i0, capacity, s);
  }
  return cuda_status(e);
}

extern "C" vio_status vio_track_patches(vio_ctx* ctx, const vio_pyr_layout* layout,
                                        const vio_pyr_batch* src, const vio_pyr_batch* dst,
                                        const float* d_pts, const float* d_init,
                                        const int32_t* d_count, int32_t capacity, int32_t flags,
                                        float* d_out, uint8_t* d_status, float* d_fb_dist,
                                        float* d_last_step, void* stream) {
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
                                       (cudaStream_t)stream, false, d_last_step));
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

extern "C" vio_status vio_match_cameras(vio_ctx* ctx, const vio_pyr_layout* layout,
                                        const vio_pyr_batch* src, const vio_pyr_batch* dst,
                                        const float* d_pts, const float* d_init,
                                        const int32_t* d_count, int32_t capacity,
                                        float* d_match, uint8_t* d_status, float* d_fb_dist,
                                        void* stream) {
  if (!ctx || !layout_ok(layout) || !batch_ok(layout, src) || !batch_ok(layout, dst))
    return VIO_ERR_INVALID_ARG;
  if (src->n_images != 1 || !d_pts || !d_match || !d_status || capacity < 0)
    return VIO_ERR_INVALID_ARG;
  // the one source image, once per target: zero strides
  vio::Batch s = vio::make_batch(*src);
  s.l0_stride = 0;
  s.upper_stride = 0;
  s.n = dst->n_images;
  vio::TrackCfg cfg{ctx->p.gn_iters, 1, ctx->p.fb_max_dist, -1};
  return cuda_status(vio::launch_track(vio::make_geom(*layout), s, vio::make_batch(*dst), d_pts,
                                       d_init, d_count, capacity, cfg, nullptr, d_match,
                                       d_status, d_fb_dist, (cudaStream_t)stream, true));
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
