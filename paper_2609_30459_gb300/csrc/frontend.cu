// Per-frame frontend state and driver (Sec. III-B): n_streams stereo streams
// of one size, all state resident on the device, nothing synchronised with
// the host inside a step. The kernels of one frame are in frame.cu.
//
// Keypoint lists, per (stream, camera), in stable order:
//   camera 0: surviving tracks, then this step's new detections
//             (cell raster order, ids next_id + rank);
//   camera 1: surviving tracks, then the new detections whose stereo match
//             passed the forward-backward check, at the matched position.
// A track survives a step if its temporal track has status OK. Detection
// counts, per cell, the surviving camera-0 tracks against k.
#include <array>
#include <new>
#include <vector>

#include "detect_dev.cuh"
#include "frame.cuh"

struct vio_frontend {
  vio_params p;
  int w, h, n_streams, capacity;
  int gx, gy;
  vio_pyr_layout layout;
  // device buffers (one allocation)
  void* d_mem;
  uint8_t* pyr[3];            // upper buffers, 2*n_streams images each, ring of 3 frames
                              // (a step's front may run while the previous step tracks
                              // between the two slots before it)
  float* list_xy;             // float2 per slot, [parity][stream][camera] x capacity
  int32_t* list_id;
  int32_t* list_count;        // [parity][stream][camera]
  uint8_t* list_status;
  float* trk_xy;              // temporal track result, float2 per slot
  uint8_t* trk_status;
  unsigned long long* cand[2];   // n_streams * cells * k candidate keys, per step parity
  int32_t* cand_count[2];        // n_streams * cells
  float* spec_xy;             // stereo matches of the candidates
  uint8_t* spec_status;
  uint8_t* occupancy;         // n_streams * cells
  float* new_xy[2];           // n_streams * capacity, per output list parity
  int32_t* new_count[2];      // n_streams, per output list parity
  int32_t* next_id;           // n_streams
  int32_t* stats;             // VIO_STATS_RING * n_streams * VIO_N_STATS
  int32_t* step_ctr;          // device count of launched steps, then its copy per parity
  float* net_out;             // flow proposals, [stream][camera] x capacity x 3
  uint8_t* trk_learned;       // per slot: tracked from the proposal
  const void* net;            // packed initializer weights (null: off)
  vio_initnet_cfg net_cfg;
  vio::FrameTune tune;        // launch shapes (the frontend keeps the frame order)
  // host state
  int cur_list;
  int cur_pyr, prev_pyr;
  cudaStream_t side = nullptr;   // fronts of pipelined steps (vio_frontend_run), low priority
  cudaStream_t main_s = nullptr; // the rest of those steps, high priority (the critical path)
  cudaStream_t copy_s = nullptr; // read-back of pipelined host steps
  cudaEvent_t ev_copied[2] = {}; // read-back of the step of this parity done
  cudaEvent_t ev_entry = nullptr, ev_exit = nullptr, ev_front[2] = {}, ev_back[3] = {};
  cudaEvent_t ev_caller = nullptr;   // the last work enqueued on a caller's stream
  bool caller_pending = false;       // the internal streams must wait for ev_caller
  bool internal_pending = false;     // a caller's stream must wait for ev_exit
  bool have_prev;
  const uint8_t* prev_frames;
  int32_t prev_pitch;
  int64_t prev_stride;
  int64_t steps;
  int timing;   // 0 off, 1 every stage boundary, 2 first and last event of a step
  std::vector<cudaEvent_t> ev_free;
  std::vector<std::array<cudaEvent_t, VIO_N_STAGES + 1>> ev_rec;
};

namespace {
size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

bool frontend_params_ok(const vio_params* p) {
  if (!p || p->n_levels < 1 || p->n_levels > VIO_MAX_LEVELS) return false;
  if (p->round_mode != 0 && p->round_mode != 1) return false;
  if (p->gn_iters < 0 || p->gn_iters > 1000 || p->pattern_id != 0) return false;
  if (p->cell_w < 1 || p->cell_h < 1 || p->cell_w > 512 || p->cell_h > 512) return false;
  if (p->k_per_cell < 1 || p->k_per_cell > VIO_MAX_K) return false;
  if (p->n_thresholds < 1 || p->n_thresholds > VIO_MAX_THRESHOLDS) return false;
  for (int i = 0; i < p->n_thresholds; ++i) {
    if (p->thresholds[i] < 0 || p->thresholds[i] > 254) return false;
    if (i > 0 && p->thresholds[i] > p->thresholds[i - 1]) return false;
  }
  return p->detect_border >= 0 && p->fb_max_dist >= 0.f;
}

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

extern "C" vio_status vio_frontend_create(vio_frontend** out, const vio_params* p, int32_t w,
                                          int32_t h, int32_t n_streams, int32_t capacity) {
  // capacity < 2^15: the finalize kernel packs two per-camera counts in one int
  if (!out || !frontend_params_ok(p) || w <= 0 || h <= 0 || n_streams <= 0 || capacity <= 0 ||
      n_streams > 65535 || capacity > 32767)
    return VIO_ERR_INVALID_ARG;
  *out = nullptr;
  vio_pyr_layout L;
  vio_status st = vio_pyr_layout_make(w, h, p->n_levels, w, &L);
  if (st != VIO_OK) return st;
  const int gx = w / p->cell_w, gy = h / p->cell_h;
  const long long n_cells = (long long)gx * gy;
  if (n_cells * p->k_per_cell > capacity) return VIO_ERR_INVALID_ARG;
  if (n_cells * 4 > 200 * 1024) return VIO_ERR_UNSUPPORTED;   // finalize's shared counters
  if (!vio::det::detect_fits(p->cell_w, p->cell_h, p->k_per_cell))
    return VIO_ERR_UNSUPPORTED;
  vio_frontend* fe = new (std::nothrow) vio_frontend();
  if (!fe) return VIO_ERR_OOM;
  fe->p = *p;
  fe->w = w;
  fe->h = h;
  fe->n_streams = n_streams;
  fe->capacity = capacity;
  fe->gx = gx;
  fe->gy = gy;
  fe->layout = L;
  const size_t nl = (size_t)2 * n_streams, slots = nl * capacity;
  const size_t ns = (size_t)n_streams, nc = (size_t)n_cells, kk = (size_t)p->k_per_cell;
  const size_t sizes[] = {
      (size_t)L.upper_bytes * nl * 3,                           // 0 pyr (ring of 3)
      0,                                                        // 1 (unused)
      2 * slots * 8,                                            // 2 list_xy
      2 * slots * 4,                                            // 3 list_id
      2 * nl * 4,                                               // 4 list_count
      2 * slots,                                                // 5 list_status
      16,                                                       // 6 step_ctr
      slots * 12,                                               // 7 net_out
      slots,                                                    // 8 trk_learned
      slots * 8, slots,                                         // 9-10 trk
      2 * ns * nc * kk * 8, 2 * ns * nc * 4,                    // 11-12 cand (2 parities)
      ns * nc * kk * 8, ns * nc * kk,                           // 13-14 spec
      ns * nc,                                                  // 15 occupancy
      2 * ns * capacity * 8, 2 * ns * 4,                        // 16-17 new (2 parities)
      ns * 4,                                                   // 18 next_id
      (size_t)VIO_STATS_RING * ns * VIO_N_STATS * 4};           // 19 stats
  constexpr size_t kN = sizeof(sizes) / sizeof(sizes[0]);
  size_t total = 0;
  for (size_t s : sizes) total += align256(s);
  if (cudaMalloc(&fe->d_mem, total) != cudaSuccess) {
    cudaGetLastError();
    delete fe;
    return VIO_ERR_OOM;
  }
  uint8_t* q = (uint8_t*)fe->d_mem;
  void* ptrs[kN];
  for (size_t i = 0; i < kN; ++i) {
    ptrs[i] = q;
    q += align256(sizes[i]);
  }
  for (int i = 0; i < 3; ++i) fe->pyr[i] = (uint8_t*)ptrs[0] + (size_t)i * L.upper_bytes * nl;
  fe->list_xy = (float*)ptrs[2];
  fe->list_id = (int32_t*)ptrs[3];
  fe->list_count = (int32_t*)ptrs[4];
  fe->list_status = (uint8_t*)ptrs[5];
  fe->step_ctr = (int32_t*)ptrs[6];
  fe->net_out = (float*)ptrs[7];
  fe->trk_learned = (uint8_t*)ptrs[8];
  fe->net = nullptr;
  fe->net_cfg = vio_initnet_cfg{};
  fe->tune = vio::FrameTune{128, 0, 0, 0, 256};
  fe->trk_xy = (float*)ptrs[9];
  fe->trk_status = (uint8_t*)ptrs[10];
  for (int i = 0; i < 2; ++i) {
    fe->cand[i] = (unsigned long long*)ptrs[11] + (size_t)i * ns * nc * kk;
    fe->cand_count[i] = (int32_t*)ptrs[12] + (size_t)i * ns * nc;
  }
  fe->spec_xy = (float*)ptrs[13];
  fe->spec_status = (uint8_t*)ptrs[14];
  fe->occupancy = (uint8_t*)ptrs[15];
  for (int i = 0; i < 2; ++i) {
    fe->new_xy[i] = (float*)ptrs[16] + (size_t)i * ns * capacity * 2;
    fe->new_count[i] = (int32_t*)ptrs[17] + (size_t)i * ns;
  }
  fe->next_id = (int32_t*)ptrs[18];
  fe->stats = (int32_t*)ptrs[19];
  if (cudaMemset(fe->d_mem, 0, total) != cudaSuccess ||
      cudaMemset(fe->list_status, VIO_TRACK_EMPTY, 2 * slots) != cudaSuccess ||
      cudaDeviceSynchronize() != cudaSuccess) {
    cudaGetLastError();
    cudaFree(fe->d_mem);
    delete fe;
    return VIO_ERR_CUDA;
  }
  fe->cur_list = 0;
  fe->cur_pyr = 0;
  fe->prev_pyr = 0;
  fe->have_prev = false;
  fe->prev_frames = nullptr;
  fe->prev_pitch = 0;
  fe->prev_stride = 0;
  fe->steps = 0;
  fe->timing = 0;
  *out = fe;
  return VIO_OK;
}

extern "C" vio_status vio_frontend_destroy(vio_frontend* fe) {
  if (!fe) return VIO_ERR_INVALID_ARG;
  for (auto& row : fe->ev_rec)
    for (cudaEvent_t e : row) cudaEventDestroy(e);
  for (cudaEvent_t e : fe->ev_free) cudaEventDestroy(e);
  if (fe->side) {
    cudaStreamSynchronize(fe->side);
    cudaStreamSynchronize(fe->main_s);
    cudaStreamSynchronize(fe->copy_s);
    cudaStreamDestroy(fe->side);
    cudaStreamDestroy(fe->main_s);
    cudaStreamDestroy(fe->copy_s);
    for (cudaEvent_t e : fe->ev_copied) cudaEventDestroy(e);
    cudaEventDestroy(fe->ev_entry);
    cudaEventDestroy(fe->ev_exit);
    cudaEventDestroy(fe->ev_caller);
    for (cudaEvent_t e : fe->ev_front) cudaEventDestroy(e);
    for (cudaEvent_t e : fe->ev_back) cudaEventDestroy(e);
  }
  cudaFree(fe->d_mem);
  delete fe;
  return VIO_OK;
}

namespace {
bool caller_enter(vio_frontend* fe, cudaStream_t s);
bool caller_leave(vio_frontend* fe, cudaStream_t s);
}  // namespace

extern "C" vio_status vio_frontend_reset(vio_frontend* fe, void* stream) {
  if (!fe) return VIO_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  if (!caller_enter(fe, s)) return VIO_ERR_CUDA;
  const size_t nl = (size_t)2 * fe->n_streams;
  cudaMemsetAsync(fe->list_count, 0, 2 * nl * 4, s);
  cudaMemsetAsync(fe->list_status, VIO_TRACK_EMPTY, 2 * nl * fe->capacity, s);
  cudaMemsetAsync(fe->next_id, 0, (size_t)fe->n_streams * 4, s);
  fe->have_prev = false;
  if (!caller_leave(fe, s)) return VIO_ERR_CUDA;
  return cudaGetLastError() == cudaSuccess ? VIO_OK : VIO_ERR_CUDA;
}

extern "C" int32_t vio_frontend_launches_per_step(const vio_frontend* fe) {
  if (!fe) return 0;
  vio_pyr_layout L;
  if (vio_pyr_layout_make(fe->w, fe->h, fe->p.n_levels, fe->w, &L) != VIO_OK) return 0;
  const vio::Geom g = vio::make_geom(L);
  return vio::frame_launches(&g, 1, fe->net != nullptr, false, fe->tune.pyr_first);
}

extern "C" vio_status vio_frontend_set_tune(vio_frontend* fe, const vio_batch_tune* t) {
  if (!fe || !t) return VIO_ERR_INVALID_ARG;
  if (t->k2_threads != 32 && t->k2_threads != 64 && t->k2_threads != 128 &&
      t->k2_threads != 256 && t->k2_threads != 512)
    return VIO_ERR_INVALID_ARG;
  if (t->pyr_tile_shift < -1 || t->pyr_tile_shift > 1 || t->stereo_after_select != 0 ||
      t->pyr_first_levels < 0 || t->pyr_first_levels > 4 ||
      (t->k1_threads != 128 && t->k1_threads != 256) ||
      (t->det_warps != 0 && t->det_warps != 1 && t->det_warps != 2 && t->det_warps != 4 &&
       t->det_warps != 8))
    return VIO_ERR_INVALID_ARG;
  fe->tune = vio::FrameTune{t->k2_threads, t->pyr_tile_shift, 0, t->pyr_first_levels,
                            t->k1_threads, t->det_warps};
  return VIO_OK;
}

extern "C" vio_status vio_frontend_set_initnet(vio_frontend* fe, const void* d_packed,
                                               const vio_initnet_cfg* cfg) {
  if (!fe) return VIO_ERR_INVALID_ARG;
  if (d_packed) {
    if (!vio::initnet_cfg_ok(cfg, fe->p.n_levels, d_packed)) return VIO_ERR_INVALID_ARG;
    if (2 * fe->n_streams > vio::KN_MAX_LISTS) return VIO_ERR_UNSUPPORTED;
    fe->net_cfg = *cfg;
  }
  fe->net = d_packed;
  return VIO_OK;
}

namespace {

// The launch description of the frontend's next step on frames d_frames
// (pyramid ring slot, candidate buffers and step-count copy of its parity).
vio_status next_launch(vio_frontend* fe, const uint8_t* d_frames, int32_t pitch,
                       int64_t frame_stride, vio::FrameLaunch& f) {
  using namespace vio;
  if (!fe || !d_frames || pitch < fe->w || frame_stride < (int64_t)pitch * fe->h)
    return VIO_ERR_INVALID_ARG;
  if (fe->have_prev && fe->prev_pitch != pitch) return VIO_ERR_UNSUPPORTED;
  const int ns = fe->n_streams;
  vio_pyr_layout L;
  vio_status st = vio_pyr_layout_make(fe->w, fe->h, fe->p.n_levels, pitch, &L);
  if (st != VIO_OK) return st;
  const long long ub = L.upper_bytes;
  const int par = (int)(fe->steps & 1);
  f = FrameLaunch{};
  f.p = fe->p;
  f.g = make_geom(L);
  f.n_streams = ns;
  f.cap = fe->capacity;
  f.cur = Batch{d_frames, frame_stride, fe->pyr[fe->cur_pyr], ub, 2 * ns};
  f.prev = fe->have_prev
               ? Batch{fe->prev_frames, fe->prev_stride, fe->pyr[fe->prev_pyr], ub, 2 * ns}
               : f.cur;
  f.slotted = 0;
  f.host_parity = fe->cur_list;
  f.host_have_prev = fe->have_prev ? 1 : 0;
  f.list_xy = fe->list_xy;
  f.list_id = fe->list_id;
  f.list_count = fe->list_count;
  f.list_status = fe->list_status;
  f.trk_xy = fe->trk_xy;
  f.trk_status = fe->trk_status;
  f.cand = fe->cand[par];
  f.cand_count = fe->cand_count[par];
  f.spec_xy = fe->spec_xy;
  f.spec_status = fe->spec_status;
  f.new_xy = fe->new_xy[fe->cur_list ^ 1];       // the step's output parity
  f.new_count = fe->new_count[fe->cur_list ^ 1];
  f.next_id = fe->next_id;
  f.occupancy = fe->occupancy;
  f.stats = fe->stats;
  f.step_ctr = fe->step_ctr;
  f.ctr_copy = fe->step_ctr + 1 + par;
  if (fe->net) {
    f.net = fe->net;
    f.net_la = fe->net_cfg.level_a;
    f.net_lb = fe->net_cfg.level_b;
    f.net_top = fe->net_cfg.start_level;
    f.net_tau = fe->net_cfg.min_conf;
    f.net_max_step = fe->net_cfg.max_last_step;
    f.net_out = fe->net_out;
    f.trk_learned = fe->trk_learned;
  }
  return VIO_OK;
}

// Host state after a step on frames d_frames has been enqueued.
void advance(vio_frontend* fe, const uint8_t* d_frames, int32_t pitch, int64_t frame_stride) {
  fe->cur_list ^= 1;
  fe->prev_pyr = fe->cur_pyr;
  fe->cur_pyr = (fe->cur_pyr + 1) % 3;
  fe->have_prev = true;
  fe->prev_frames = d_frames;
  fe->prev_pitch = pitch;
  fe->prev_stride = frame_stride;
  ++fe->steps;
}

// Internal streams of pipelined steps (created once): the fronts on a
// low-priority stream, the rest on a high-priority one (the critical path).
bool ensure_pipe(vio_frontend* fe) {
  if (fe->side) return true;
  int least = 0, greatest = 0;
  if (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess ||
      cudaStreamCreateWithPriority(&fe->side, cudaStreamNonBlocking, least) != cudaSuccess ||
      cudaStreamCreateWithPriority(&fe->main_s, cudaStreamNonBlocking, greatest) != cudaSuccess ||
      cudaStreamCreateWithFlags(&fe->copy_s, cudaStreamNonBlocking) != cudaSuccess)
    return false;
  cudaEvent_t* evs[] = {&fe->ev_entry,    &fe->ev_exit,     &fe->ev_caller,
                        &fe->ev_front[0], &fe->ev_front[1], &fe->ev_back[0],
                        &fe->ev_back[1],  &fe->ev_back[2],  &fe->ev_copied[0],
                        &fe->ev_copied[1]};
  for (cudaEvent_t* e : evs)
    if (cudaEventCreateWithFlags(e, cudaEventDisableTiming) != cudaSuccess) return false;
  return true;
}

// Work on a caller's stream s follows the frontend's pipelined steps, and
// pipelined steps follow work on a caller's stream.
bool caller_enter(vio_frontend* fe, cudaStream_t s) {
  if (fe->internal_pending) {
    if (cudaStreamWaitEvent(s, fe->ev_exit, 0) != cudaSuccess) return false;
    fe->internal_pending = false;
  }
  return true;
}
bool caller_leave(vio_frontend* fe, cudaStream_t s) {
  if (!fe->side) return true;   // no pipelined step yet: nothing to order
  if (cudaEventRecord(fe->ev_caller, s) != cudaSuccess) return false;
  fe->caller_pending = true;
  return true;
}
bool internal_enter(vio_frontend* fe) {
  if (fe->caller_pending) {
    if (cudaStreamWaitEvent(fe->side, fe->ev_caller, 0) != cudaSuccess ||
        cudaStreamWaitEvent(fe->main_s, fe->ev_caller, 0) != cudaSuccess ||
        cudaStreamWaitEvent(fe->copy_s, fe->ev_caller, 0) != cudaSuccess)
      return false;
    fe->caller_pending = false;
  }
  return true;
}

// One pipelined step on the internal streams: optional upload (h_frames ->
// d_frames) and front on the low-priority stream, after the end of the step
// two back; the rest on the high-priority stream; then ev_back of this step.
vio_status pipelined_step(vio_frontend* fe, const uint8_t* h_frames, const uint8_t* d_frames,
                          int32_t pitch, int64_t frame_stride) {
  using namespace vio;
  FrameLaunch f;
  const vio_status st = next_launch(fe, d_frames, pitch, frame_stride, f);
  if (st != VIO_OK) return st;
  const int64_t t = fe->steps;
  if (t >= 2 && cudaStreamWaitEvent(fe->side, fe->ev_back[(t - 2) % 3], 0) != cudaSuccess)
    return VIO_ERR_CUDA;
  if (h_frames && cudaMemcpyAsync(const_cast<uint8_t*>(d_frames), h_frames,
                                  (size_t)2 * fe->n_streams * frame_stride,
                                  cudaMemcpyHostToDevice, fe->side) != cudaSuccess)
    return VIO_ERR_CUDA;
  // the lists this step writes were read back (if at all) after step t-2
  if (t >= 2 && cudaStreamWaitEvent(fe->main_s, fe->ev_copied[t % 2], 0) != cudaSuccess)
    return VIO_ERR_CUDA;
  if (launch_frames(&f, 1, fe->tune, fe->side, nullptr, 1) != cudaSuccess ||
      cudaEventRecord(fe->ev_front[t % 2], fe->side) != cudaSuccess ||
      cudaStreamWaitEvent(fe->main_s, fe->ev_front[t % 2], 0) != cudaSuccess ||
      launch_frames(&f, 1, fe->tune, fe->main_s, nullptr, 2) != cudaSuccess ||
      cudaEventRecord(fe->ev_back[t % 3], fe->main_s) != cudaSuccess)
    return VIO_ERR_CUDA;
  advance(fe, d_frames, pitch, frame_stride);
  return VIO_OK;
}

}  // namespace

extern "C" vio_status vio_frontend_step(vio_frontend* fe, const uint8_t* d_frames,
                                        int32_t pitch, int64_t frame_stride, void* stream) {
  using namespace vio;
  FrameLaunch f;
  const vio_status st = next_launch(fe, d_frames, pitch, frame_stride, f);
  if (st != VIO_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  if (!caller_enter(fe, s)) return VIO_ERR_CUDA;
  std::array<cudaEvent_t, VIO_N_STAGES + 1> ev{};
  if (fe->timing)
    for (int i = 0; i <= VIO_N_STAGES; ++i)
      if ((fe->timing == 1 || i == 0 || i == VIO_N_STAGES) && !(ev[i] = take_event(fe)))
        return VIO_ERR_CUDA;
  if (launch_frames(&f, 1, fe->tune, s, fe->timing ? ev.data() : nullptr) != cudaSuccess)
    return VIO_ERR_CUDA;
  if (fe->timing) fe->ev_rec.push_back(ev);
  advance(fe, d_frames, pitch, frame_stride);
  return caller_leave(fe, s) ? VIO_OK : VIO_ERR_CUDA;
}

namespace {

// Lists and new detections of the last step into pinned host buffers.
bool copy_outputs(vio_frontend* fe, float* h_track_xy, int32_t* h_track_id,
                  int32_t* h_track_count, float* h_new_xy, int32_t* h_new_count,
                  cudaStream_t s) {
  vio_frontend_view v;
  vio_frontend_get_view(fe, &v);
  const size_t nl = (size_t)2 * fe->n_streams, cap = fe->capacity;
  return cudaMemcpyAsync(h_track_xy, v.d_track_xy, nl * cap * 8, cudaMemcpyDeviceToHost, s) ==
             cudaSuccess &&
         cudaMemcpyAsync(h_track_id, v.d_track_id, nl * cap * 4, cudaMemcpyDeviceToHost, s) ==
             cudaSuccess &&
         cudaMemcpyAsync(h_track_count, v.d_track_count, nl * 4, cudaMemcpyDeviceToHost, s) ==
             cudaSuccess &&
         cudaMemcpyAsync(h_new_xy, v.d_new_xy, (size_t)fe->n_streams * cap * 8,
                         cudaMemcpyDeviceToHost, s) == cudaSuccess &&
         cudaMemcpyAsync(h_new_count, v.d_new_count, (size_t)fe->n_streams * 4,
                         cudaMemcpyDeviceToHost, s) == cudaSuccess;
}

bool host_args_ok(const vio_frontend* fe, const uint8_t* h_frames, const uint8_t* d_frames,
                  int32_t pitch, int64_t frame_stride, const void* a, const void* b,
                  const void* c, const void* d, const void* e) {
  return fe && h_frames && d_frames && a && b && c && d && e && pitch >= fe->w &&
         frame_stride >= (int64_t)pitch * fe->h;
}

}  // namespace

extern "C" vio_status vio_frontend_step_host(vio_frontend* fe, const uint8_t* h_frames,
                                             uint8_t* d_frames, int32_t pitch,
                                             int64_t frame_stride, float* h_track_xy,
                                             int32_t* h_track_id, int32_t* h_track_count,
                                             float* h_new_xy, int32_t* h_new_count,
                                             void* stream) {
  if (!host_args_ok(fe, h_frames, d_frames, pitch, frame_stride, h_track_xy, h_track_id,
                    h_track_count, h_new_xy, h_new_count))
    return VIO_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  if (!caller_enter(fe, s)) return VIO_ERR_CUDA;
  const size_t in_bytes = (size_t)2 * fe->n_streams * frame_stride;
  if (cudaMemcpyAsync(d_frames, h_frames, in_bytes, cudaMemcpyHostToDevice, s) != cudaSuccess)
    return VIO_ERR_CUDA;
  const vio_status st = vio_frontend_step(fe, d_frames, pitch, frame_stride, stream);
  if (st != VIO_OK) return st;
  if (!copy_outputs(fe, h_track_xy, h_track_id, h_track_count, h_new_xy, h_new_count, s))
    return VIO_ERR_CUDA;
  return caller_leave(fe, s) ? VIO_OK : VIO_ERR_CUDA;
}

extern "C" vio_status vio_frontend_step_host_async(vio_frontend* fe, const uint8_t* h_frames,
                                                   uint8_t* d_frames, int32_t pitch,
                                                   int64_t frame_stride, float* h_track_xy,
                                                   int32_t* h_track_id, int32_t* h_track_count,
                                                   float* h_new_xy, int32_t* h_new_count,
                                                   void* done_event) {
  if (!host_args_ok(fe, h_frames, d_frames, pitch, frame_stride, h_track_xy, h_track_id,
                    h_track_count, h_new_xy, h_new_count))
    return VIO_ERR_INVALID_ARG;
  if (fe->timing) return VIO_ERR_UNSUPPORTED;   // stage timing keeps steps whole
  if (!ensure_pipe(fe) || !internal_enter(fe)) return VIO_ERR_CUDA;
  const int64_t t = fe->steps;
  const vio_status st = pipelined_step(fe, h_frames, d_frames, pitch, frame_stride);
  if (st != VIO_OK) return st;
  // read-back beside the next step's tracking, before the step after it
  // overwrites these lists
  if (cudaStreamWaitEvent(fe->copy_s, fe->ev_back[t % 3], 0) != cudaSuccess ||
      !copy_outputs(fe, h_track_xy, h_track_id, h_track_count, h_new_xy, h_new_count,
                    fe->copy_s) ||
      cudaEventRecord(fe->ev_copied[t % 2], fe->copy_s) != cudaSuccess ||
      (done_event && cudaEventRecord((cudaEvent_t)done_event, fe->copy_s) != cudaSuccess) ||
      cudaEventRecord(fe->ev_exit, fe->copy_s) != cudaSuccess)
    return VIO_ERR_CUDA;
  fe->internal_pending = true;
  return VIO_OK;
}

extern "C" vio_status vio_frontend_run(vio_frontend* fe, const uint8_t* d_frames, int32_t pitch,
                                       int64_t frame_stride, int64_t step_stride,
                                       int32_t n_steps, void* stream) {
  using namespace vio;
  if (!fe || !d_frames || n_steps < 0 || step_stride < 0) return VIO_ERR_INVALID_ARG;
  if (n_steps > 1 && step_stride < (int64_t)2 * fe->n_streams * frame_stride)
    return VIO_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  // Pipelined steps: the front of step t (pyramids and detection candidates
  // of its own frames) runs on a low-priority stream beside the tracking and
  // finalisation of step t-1 (on a high-priority stream: the critical path);
  // it waits for the end of step t-2, the last reader of its pyramid ring
  // slot and candidate buffers. The run follows the work already on the
  // caller's stream, and the caller's stream waits for its last step. Stage
  // timing keeps the steps whole.
  if (n_steps < 2 || fe->timing) {
    for (int32_t i = 0; i < n_steps; ++i) {
      const vio_status st =
          vio_frontend_step(fe, d_frames + (int64_t)i * step_stride, pitch, frame_stride, stream);
      if (st != VIO_OK) return st;
    }
    return VIO_OK;
  }
  if (!ensure_pipe(fe) || !caller_enter(fe, s) ||
      cudaEventRecord(fe->ev_caller, s) != cudaSuccess)
    return VIO_ERR_CUDA;
  fe->caller_pending = true;
  if (!internal_enter(fe)) return VIO_ERR_CUDA;
  for (int32_t i = 0; i < n_steps; ++i) {
    const vio_status st =
        pipelined_step(fe, nullptr, d_frames + (int64_t)i * step_stride, pitch, frame_stride);
    if (st != VIO_OK) return st;
  }
  if (cudaEventRecord(fe->ev_exit, fe->main_s) != cudaSuccess ||
      cudaStreamWaitEvent(s, fe->ev_exit, 0) != cudaSuccess)
    return VIO_ERR_CUDA;
  fe->internal_pending = false;
  return VIO_OK;
}

extern "C" vio_status vio_frontend_set_timing(vio_frontend* fe, int32_t enable) {
  if (!fe) return VIO_ERR_INVALID_ARG;
  if (enable < 0 || enable > 2) return VIO_ERR_INVALID_ARG;
  fe->timing = enable;
  return VIO_OK;
}

extern "C" vio_status vio_frontend_read_timing(vio_frontend* fe, double* stage_ms,
                                               int64_t* n_steps, float* step_ms,
                                               int64_t step_ms_cap) {
  if (!fe || !stage_ms || !n_steps) return VIO_ERR_INVALID_ARG;
  for (int i = 0; i < VIO_N_STAGES; ++i) stage_ms[i] = 0.0;
  vio_status st = VIO_OK;
  int64_t k = 0;
  for (auto& row : fe->ev_rec) {
    if (cudaEventSynchronize(row[VIO_N_STAGES]) != cudaSuccess) st = VIO_ERR_CUDA;
    for (int i = 0; i < VIO_N_STAGES; ++i) {
      float ms = 0.f;
      if (row[i] && row[i + 1] && cudaEventElapsedTime(&ms, row[i], row[i + 1]) == cudaSuccess)
        stage_ms[i] += ms;
    }
    if (step_ms && k < step_ms_cap) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, row[0], row[VIO_N_STAGES]);
      step_ms[k] = ms;
    }
    ++k;
    for (cudaEvent_t e : row)
      if (e) fe->ev_free.push_back(e);
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
  const size_t nl = (size_t)2 * fe->n_streams, li = (size_t)fe->cur_list;
  out->d_track_xy = fe->list_xy + 2 * li * nl * fe->capacity;
  out->d_track_id = fe->list_id + li * nl * fe->capacity;
  out->d_track_status = fe->list_status + li * nl * fe->capacity;
  out->d_track_count = fe->list_count + li * nl;
  out->d_new_xy = fe->new_xy[li];
  out->d_new_count = fe->new_count[li];
  out->capacity = fe->capacity;
  out->n_streams = fe->n_streams;
  return VIO_OK;
}
