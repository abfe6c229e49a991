// Per-frame frontend (Sec. III-B): stage order pyramid -> temporal tracking
// -> detection -> cross-camera matching, for n_streams stereo streams of one
// size, with all state resident on the device and nothing synchronised with
// the host inside a step.
//
// Keypoint lists, per (stream, camera), in stable order:
//   camera 0: surviving tracks, then this step's new detections
//             (cell raster order, ids next_id + rank);
//   camera 1: surviving tracks, then the new detections whose stereo match
//             passed the forward-backward check, at the matched position.
// A track survives a step if its temporal track has status OK. Detection
// counts, per cell, the surviving camera-0 tracks against k.
#include <stdlib.h>

#include <array>
#include <new>
#include <vector>

#include "common.cuh"

namespace vio {
namespace {

constexpr int CMP_THREADS = 256;

// cell index of a position, exact: the largest cx with cx * cw <= x
__device__ __forceinline__ int cell_of(float x, int cw) {
  int c = (int)floorf(x / (float)cw);
  if ((float)(c + 1) * (float)cw <= x) ++c;
  if ((float)c * (float)cw > x) --c;
  return c;
}

// One CTA per (stream, camera): keep the slots whose status is OK, in order.
// Camera 0 also counts survivors per detection cell (saturating at 255).
__global__ void __launch_bounds__(CMP_THREADS) compact_kernel(
    const float* __restrict__ pos, const uint8_t* __restrict__ status,
    const int32_t* __restrict__ ids_in, const int32_t* __restrict__ count_in, int capacity,
    float* __restrict__ pos_out, int32_t* __restrict__ ids_out, int32_t* __restrict__ count_out,
    uint8_t* __restrict__ occupancy, int gx, int gy, int cw, int ch,
    int32_t* __restrict__ stats) {
  extern __shared__ int occ_s[];
  __shared__ int warp_sums[CMP_THREADS / 32];
  __shared__ int carry_s;
  const int list = blockIdx.x;           // 2 * stream + camera
  const bool cam0 = (list & 1) == 0;
  const int stream = list >> 1;
  const int n_cells = gx * gy;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (cam0)
    for (int i = threadIdx.x; i < n_cells; i += CMP_THREADS) occ_s[i] = 0;
  if (threadIdx.x == 0) carry_s = 0;
  __syncthreads();
  const long long base = (long long)list * capacity;
  const int n = min(count_in[list], capacity);
  for (int c0 = 0; c0 < n; c0 += CMP_THREADS) {
    const int i = c0 + threadIdx.x;
    const int keep = (i < n && status[base + i] == VIO_TRACK_OK) ? 1 : 0;
    int incl = keep;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    if (lane == 31) warp_sums[warp] = incl;
    __syncthreads();
    if (warp == 0) {
      int ws = lane < CMP_THREADS / 32 ? warp_sums[lane] : 0;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, ws, o);
        if (lane >= o) ws += t;
      }
      if (lane < CMP_THREADS / 32) warp_sums[lane] = ws;
    }
    __syncthreads();
    const int carry = carry_s;
    if (keep) {
      const int o = carry + (warp ? warp_sums[warp - 1] : 0) + incl - 1;
      const float x = pos[2 * (base + i)], y = pos[2 * (base + i) + 1];
      pos_out[2 * (base + o)] = x;
      pos_out[2 * (base + o) + 1] = y;
      ids_out[base + o] = ids_in[base + i];
      if (cam0 && x >= 0.f && y >= 0.f) {
        const int cx = cell_of(x, cw), cy = cell_of(y, ch);
        if (cx < gx && cy < gy) atomicAdd(&occ_s[cy * gx + cx], 1);
      }
    }
    __syncthreads();
    if (threadIdx.x == CMP_THREADS - 1) carry_s = carry + warp_sums[CMP_THREADS / 32 - 1];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    count_out[list] = carry_s;
    stats[stream * VIO_N_STATS + VIO_STAT_TRK0 + (list & 1)] = n;
    stats[stream * VIO_N_STATS + VIO_STAT_OK0 + (list & 1)] = carry_s;
  }
  if (cam0)
    for (int i = threadIdx.x; i < n_cells; i += CMP_THREADS)
      occupancy[(long long)stream * n_cells + i] = (uint8_t)min(occ_s[i], 255);
}

// One CTA per stream: append the new detections to camera 0 and their
// successful stereo matches to camera 1; assign ids.
__global__ void __launch_bounds__(CMP_THREADS) append_kernel(
    const float* __restrict__ new_xy, const int32_t* __restrict__ new_count,
    const float* __restrict__ match_xy, const uint8_t* __restrict__ match_status,
    int capacity, float* __restrict__ pos, int32_t* __restrict__ ids,
    uint8_t* __restrict__ lstatus, int32_t* __restrict__ count, int32_t* __restrict__ next_id,
    int32_t* __restrict__ stats, int first) {
  __shared__ int warp_sums[CMP_THREADS / 32];
  __shared__ int carry_s;
  const int s = blockIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nn = min(new_count[s], capacity);
  const int id0 = next_id[s];
  const long long b0 = (long long)(2 * s) * capacity, b1 = b0 + capacity;
  const long long bn = (long long)s * capacity;
  const int c0 = count[2 * s], c1 = count[2 * s + 1];
  for (int r = threadIdx.x; r < nn; r += CMP_THREADS) {
    const int o = c0 + r;
    if (o < capacity) {
      pos[2 * (b0 + o)] = new_xy[2 * (bn + r)];
      pos[2 * (b0 + o) + 1] = new_xy[2 * (bn + r) + 1];
      ids[b0 + o] = id0 + r;
    }
  }
  if (threadIdx.x == 0) carry_s = 0;
  __syncthreads();
  for (int r0 = 0; r0 < nn; r0 += CMP_THREADS) {
    const int r = r0 + threadIdx.x;
    const int keep = (r < nn && match_status[bn + r] == VIO_TRACK_OK) ? 1 : 0;
    int incl = keep;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    if (lane == 31) warp_sums[warp] = incl;
    __syncthreads();
    if (warp == 0) {
      int ws = lane < CMP_THREADS / 32 ? warp_sums[lane] : 0;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, ws, o);
        if (lane >= o) ws += t;
      }
      if (lane < CMP_THREADS / 32) warp_sums[lane] = ws;
    }
    __syncthreads();
    const int carry = carry_s;
    if (keep) {
      const int o = c1 + carry + (warp ? warp_sums[warp - 1] : 0) + incl - 1;
      if (o < capacity) {
        pos[2 * (b1 + o)] = match_xy[2 * (bn + r)];
        pos[2 * (b1 + o) + 1] = match_xy[2 * (bn + r) + 1];
        ids[b1 + o] = id0 + r;
      }
    }
    __syncthreads();
    if (threadIdx.x == CMP_THREADS - 1) carry_s = carry + warp_sums[CMP_THREADS / 32 - 1];
    __syncthreads();
  }
  const int n0 = min(c0 + nn, capacity), n1 = min(c1 + carry_s, capacity);
  for (int i = threadIdx.x; i < capacity; i += CMP_THREADS) {
    lstatus[b0 + i] = i < n0 ? VIO_TRACK_OK : VIO_TRACK_EMPTY;
    lstatus[b1 + i] = i < n1 ? VIO_TRACK_OK : VIO_TRACK_EMPTY;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    count[2 * s] = n0;
    count[2 * s + 1] = n1;
    next_id[s] = id0 + nn;
    int32_t* st = stats + s * VIO_N_STATS;
    if (first) st[VIO_STAT_TRK0] = st[VIO_STAT_TRK1] = st[VIO_STAT_OK0] = st[VIO_STAT_OK1] = 0;
    st[VIO_STAT_NEW] = nn;
    st[VIO_STAT_MATCHED] = carry_s;
  }
}

}  // namespace
}  // namespace vio

struct vio_frontend {
  vio_params p;
  int w, h, n_streams, capacity;
  vio_pyr_layout layout;
  vio_ctx* ctx;
  int gx, gy;
  // device buffers (one allocation)
  void* d_mem;
  uint8_t* pyr[2];            // upper buffers, 2*n_streams images each, ring of 2 frames
  float* list_xy[2];          // float2 per slot, (2*n_streams) * capacity
  int32_t* list_id[2];
  int32_t* list_count[2];     // 2*n_streams
  uint8_t* list_status;       // status of the current list (output view)
  float* trk_xy;              // temporal track result, float2 per slot
  uint8_t* trk_status;
  uint8_t* occupancy;         // n_streams * n_cells
  float* new_xy;              // n_streams * capacity
  int16_t* new_score;
  int32_t* new_count;         // n_streams
  float* match_xy;            // n_streams * capacity
  uint8_t* match_status;
  int32_t* next_id;           // n_streams
  int32_t* stats;             // VIO_STATS_RING * n_streams * VIO_N_STATS
  // host state
  int64_t steps;
  bool timing;
  std::vector<cudaEvent_t> ev_free;                    // event pool
  std::vector<std::array<cudaEvent_t, VIO_N_STAGES + 1>> ev_rec;  // one row per timed step
  int cur_list;
  int cur_pyr;
  bool have_prev;
  const uint8_t* prev_frames;
  int32_t prev_pitch;
  int64_t prev_stride;
};

namespace {
size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }
}  // namespace

extern "C" vio_status vio_frontend_create(vio_frontend** out, const vio_params* p, int32_t w,
                                          int32_t h, int32_t n_streams, int32_t capacity) {
  if (!out || !p || w <= 0 || h <= 0 || n_streams <= 0 || capacity <= 0)
    return VIO_ERR_INVALID_ARG;
  *out = nullptr;
  vio_pyr_layout L;
  vio_status st = vio_pyr_layout_make(w, h, p->n_levels, w, &L);
  if (st != VIO_OK) return st;
  const int gx = w / p->cell_w, gy = h / p->cell_h;
  if ((long long)gx * gy * p->k_per_cell > capacity) return VIO_ERR_INVALID_ARG;
  vio_frontend* fe = new (std::nothrow) vio_frontend();
  if (!fe) return VIO_ERR_OOM;
  fe->p = *p;
  fe->w = w;
  fe->h = h;
  fe->n_streams = n_streams;
  fe->capacity = capacity;
  fe->layout = L;
  fe->gx = gx;
  fe->gy = gy;
  st = vio_ctx_create(&fe->ctx, p, w, h, n_streams);
  if (st != VIO_OK) {
    delete fe;
    return st;
  }
  const size_t nl = (size_t)2 * n_streams, slots = nl * capacity;
  const size_t ns = (size_t)n_streams, nc = (size_t)gx * gy;
  const size_t sizes[] = {
      (size_t)L.upper_bytes * nl, (size_t)L.upper_bytes * nl,   // pyr[0..1]
      slots * 8, slots * 8,                                     // list_xy
      slots * 4, slots * 4,                                     // list_id
      nl * 4, nl * 4,                                           // list_count
      slots,                                                    // list_status
      slots * 8, slots,                                         // trk
      ns * nc,                                                  // occupancy
      ns * capacity * 8, ns * capacity * 2, ns * 4,             // new
      ns * capacity * 8, ns * capacity,                         // match
      ns * 4,                                                   // next_id
      (size_t)VIO_STATS_RING * ns * VIO_N_STATS * 4};           // stats
  size_t total = 0;
  for (size_t s : sizes) total += align256(s);
  if (cudaMalloc(&fe->d_mem, total) != cudaSuccess) {
    cudaGetLastError();
    vio_ctx_destroy(fe->ctx);
    delete fe;
    return VIO_ERR_OOM;
  }
  uint8_t* q = (uint8_t*)fe->d_mem;
  void* ptrs[sizeof(sizes) / sizeof(sizes[0])];
  for (size_t i = 0; i < sizeof(sizes) / sizeof(sizes[0]); ++i) {
    ptrs[i] = q;
    q += align256(sizes[i]);
  }
  fe->pyr[0] = (uint8_t*)ptrs[0];
  fe->pyr[1] = (uint8_t*)ptrs[1];
  fe->list_xy[0] = (float*)ptrs[2];
  fe->list_xy[1] = (float*)ptrs[3];
  fe->list_id[0] = (int32_t*)ptrs[4];
  fe->list_id[1] = (int32_t*)ptrs[5];
  fe->list_count[0] = (int32_t*)ptrs[6];
  fe->list_count[1] = (int32_t*)ptrs[7];
  fe->list_status = (uint8_t*)ptrs[8];
  fe->trk_xy = (float*)ptrs[9];
  fe->trk_status = (uint8_t*)ptrs[10];
  fe->occupancy = (uint8_t*)ptrs[11];
  fe->new_xy = (float*)ptrs[12];
  fe->new_score = (int16_t*)ptrs[13];
  fe->new_count = (int32_t*)ptrs[14];
  fe->match_xy = (float*)ptrs[15];
  fe->match_status = (uint8_t*)ptrs[16];
  fe->next_id = (int32_t*)ptrs[17];
  fe->stats = (int32_t*)ptrs[18];
  fe->steps = 0;
  fe->timing = false;
  if (cudaMemset(fe->d_mem, 0, total) != cudaSuccess ||
      cudaMemset(fe->list_status, VIO_TRACK_EMPTY, slots) != cudaSuccess ||
      cudaDeviceSynchronize() != cudaSuccess) {
    cudaGetLastError();
    cudaFree(fe->d_mem);
    vio_ctx_destroy(fe->ctx);
    delete fe;
    return VIO_ERR_CUDA;
  }
  fe->cur_list = 0;
  fe->cur_pyr = 0;
  fe->have_prev = false;
  *out = fe;
  return VIO_OK;
}

extern "C" vio_status vio_frontend_destroy(vio_frontend* fe) {
  if (!fe) return VIO_ERR_INVALID_ARG;
  for (auto& row : fe->ev_rec)
    for (cudaEvent_t e : row) cudaEventDestroy(e);
  for (cudaEvent_t e : fe->ev_free) cudaEventDestroy(e);
  cudaFree(fe->d_mem);
  vio_ctx_destroy(fe->ctx);
  delete fe;
  return VIO_OK;
}

extern "C" vio_status vio_frontend_reset(vio_frontend* fe, void* stream) {
  if (!fe) return VIO_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t nl = (size_t)2 * fe->n_streams;
  cudaMemsetAsync(fe->list_count[0], 0, nl * 4, s);
  cudaMemsetAsync(fe->list_count[1], 0, nl * 4, s);
  cudaMemsetAsync(fe->list_status, VIO_TRACK_EMPTY, nl * fe->capacity, s);
  cudaMemsetAsync(fe->next_id, 0, (size_t)fe->n_streams * 4, s);
  fe->have_prev = false;
  return cudaGetLastError() == cudaSuccess ? VIO_OK : VIO_ERR_CUDA;
}

extern "C" int32_t vio_frontend_launches_per_step(const vio_frontend* fe) {
  if (!fe) return 0;
  // pyramid levels, temporal track, compaction, detect cells + select,
  // stereo, append
  return (fe->p.n_levels - 1) + 1 + 1 + 2 + 1 + 1;
}

namespace {
cudaEvent_t take_event(vio_frontend* fe) {
  if (!fe->ev_free.empty()) {
    cudaEvent_t e = fe->ev_free.back();
    fe->ev_free.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}
}  // namespace

extern "C" vio_status vio_frontend_step(vio_frontend* fe, const uint8_t* d_frames,
                                        int32_t pitch, int64_t frame_stride, void* stream) {
  using namespace vio;
  if (!fe || !d_frames || pitch < fe->w || frame_stride < (int64_t)pitch * fe->h)
    return VIO_ERR_INVALID_ARG;
  if (fe->have_prev && fe->prev_pitch != pitch) return VIO_ERR_UNSUPPORTED;
  cudaStream_t s = (cudaStream_t)stream;
  const int ns = fe->n_streams, cap = fe->capacity;
  vio_pyr_layout L;
  vio_status st = vio_pyr_layout_make(fe->w, fe->h, fe->p.n_levels, pitch, &L);
  if (st != VIO_OK) return st;
  const Geom g = make_geom(L);
  const long long ub = L.upper_bytes;
  const int cur = fe->cur_pyr, prv = cur ^ 1;
  const int li = fe->cur_list, lo = li ^ 1;
  const int n_cells = fe->gx * fe->gy;
  int32_t* stats = fe->stats + (fe->steps % VIO_STATS_RING) * ns * VIO_N_STATS;

  std::array<cudaEvent_t, VIO_N_STAGES + 1> ev{};
  if (fe->timing)
    for (auto& e : ev)
      if (!(e = take_event(fe))) return VIO_ERR_CUDA;
  auto mark = [&](int i) {
    if (fe->timing) cudaEventRecord(ev[i], s);
  };

  // 1. pyramids of all 2*ns images of this frame
  mark(VIO_STAGE_PYRAMID);
  Batch cur_all{d_frames, frame_stride, fe->pyr[cur], ub, 2 * ns};
  cudaError_t e = launch_pyramid(g, cur_all, fe->p.round_mode, s);
  if (e != cudaSuccess) return VIO_ERR_CUDA;

  // 2. temporal tracking with the forward-backward check, then compaction
  mark(VIO_STAGE_TRACK);
  if (fe->have_prev) {
    Batch prev_all{fe->prev_frames, fe->prev_stride, fe->pyr[prv], ub, 2 * ns};
    TrackCfg cfg{fe->p.gn_iters, 1, fe->p.fb_max_dist};
    e = launch_track(g, prev_all, cur_all, fe->list_xy[li], nullptr, fe->list_count[li], cap,
                     cfg, nullptr, fe->trk_xy, fe->trk_status, nullptr, s);
    if (e != cudaSuccess) return VIO_ERR_CUDA;
    mark(VIO_STAGE_COMPACT);
    const size_t smem = (size_t)n_cells * sizeof(int);
    if (smem > 48 * 1024) {
      e = cudaFuncSetAttribute(compact_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)smem);
      if (e != cudaSuccess) return VIO_ERR_CUDA;
    }
    compact_kernel<<<2 * ns, CMP_THREADS, smem, s>>>(
        fe->trk_xy, fe->trk_status, fe->list_id[li], fe->list_count[li], cap, fe->list_xy[lo],
        fe->list_id[lo], fe->list_count[lo], fe->occupancy, fe->gx, fe->gy, fe->p.cell_w,
        fe->p.cell_h, stats);
  } else {
    mark(VIO_STAGE_COMPACT);
    cudaMemsetAsync(fe->list_count[lo], 0, (size_t)2 * ns * 4, s);
    cudaMemsetAsync(fe->occupancy, 0, (size_t)ns * n_cells, s);
  }
  if (cudaGetLastError() != cudaSuccess) return VIO_ERR_CUDA;

  // 3. detection on camera 0 (every other image of the batch)
  mark(VIO_STAGE_DETECT);
  Batch cam0{d_frames, 2 * frame_stride, fe->pyr[cur], 2 * ub, ns};
  Batch cam1{d_frames + frame_stride, 2 * frame_stride, fe->pyr[cur] + ub, 2 * ub, ns};
  e = launch_detect(fe->p, g, cam0, fe->occupancy, nullptr, 0, fe->ctx->d_cand,
                    fe->ctx->d_cand_count, fe->new_xy, fe->new_score, fe->new_count, cap, s);
  if (e != cudaSuccess) return VIO_ERR_CUDA;

  // 4. stereo matching of the new keypoints, camera 0 -> camera 1
  mark(VIO_STAGE_STEREO);
  TrackCfg cfg{fe->p.gn_iters, 1, fe->p.fb_max_dist};
  e = launch_track(g, cam0, cam1, fe->new_xy, nullptr, fe->new_count, cap, cfg, nullptr,
                   fe->match_xy, fe->match_status, nullptr, s);
  if (e != cudaSuccess) return VIO_ERR_CUDA;

  // 5. append new keypoints and their matches
  mark(VIO_STAGE_APPEND);
  append_kernel<<<ns, CMP_THREADS, 0, s>>>(fe->new_xy, fe->new_count, fe->match_xy,
                                           fe->match_status, cap, fe->list_xy[lo],
                                           fe->list_id[lo], fe->list_status,
                                           fe->list_count[lo], fe->next_id, stats,
                                           fe->have_prev ? 0 : 1);
  mark(VIO_N_STAGES);
  if (cudaGetLastError() != cudaSuccess) return VIO_ERR_CUDA;
  if (fe->timing) fe->ev_rec.push_back(ev);

  fe->cur_list = lo;
  fe->cur_pyr = prv;
  fe->have_prev = true;
  fe->prev_frames = d_frames;
  fe->prev_pitch = pitch;
  fe->prev_stride = frame_stride;
  ++fe->steps;
  return VIO_OK;
}

extern "C" vio_status vio_frontend_set_timing(vio_frontend* fe, int32_t enable) {
  if (!fe) return VIO_ERR_INVALID_ARG;
  fe->timing = enable != 0;
  return VIO_OK;
}

extern "C" vio_status vio_frontend_read_timing(vio_frontend* fe, double* stage_ms,
                                               int64_t* n_steps) {
  if (!fe || !stage_ms || !n_steps) return VIO_ERR_INVALID_ARG;
  for (int i = 0; i < VIO_N_STAGES; ++i) stage_ms[i] = 0.0;
  vio_status st = VIO_OK;
  for (auto& row : fe->ev_rec) {
    if (cudaEventSynchronize(row[VIO_N_STAGES]) != cudaSuccess) st = VIO_ERR_CUDA;
    for (int i = 0; i < VIO_N_STAGES; ++i) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, row[i], row[i + 1]) == cudaSuccess) stage_ms[i] += ms;
    }
    for (cudaEvent_t e : row) fe->ev_free.push_back(e);
  }
  *n_steps = (int64_t)fe->ev_rec.size();
  fe->ev_rec.clear();
  cudaGetLastError();
  return st;
}

extern "C" vio_status vio_frontend_read_stats(vio_frontend* fe, int32_t* host_out,
                                              int64_t* n_steps) {
  if (!fe || !host_out || !n_steps) return VIO_ERR_INVALID_ARG;
  const size_t bytes = (size_t)VIO_STATS_RING * fe->n_streams * VIO_N_STATS * 4;
  if (cudaMemcpy(host_out, fe->stats, bytes, cudaMemcpyDeviceToHost) != cudaSuccess)
    return VIO_ERR_CUDA;
  *n_steps = fe->steps;
  return VIO_OK;
}

extern "C" vio_status vio_frontend_get_view(vio_frontend* fe, vio_frontend_view* out) {
  if (!fe || !out) return VIO_ERR_INVALID_ARG;
  const int li = fe->cur_list;
  out->d_track_xy = fe->list_xy[li];
  out->d_track_id = fe->list_id[li];
  out->d_track_status = fe->list_status;
  out->d_track_count = fe->list_count[li];
  out->d_new_xy = fe->new_xy;
  out->d_new_count = fe->new_count;
  out->capacity = fe->capacity;
  out->n_streams = fe->n_streams;
  return VIO_OK;
}
