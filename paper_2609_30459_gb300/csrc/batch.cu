// Batched multi-stream frontend (one step = the same three launches for
// every stream of every size group), with per-stream device state so that
// any subset of streams can be stepped by one captured launch sequence.
//
// Per group, device memory holds: two frame slots per stream (both cameras),
// the pyramids of both slots, keypoint lists [parity][stream][camera], the
// per-stream parity / first-frame flag / activity words, and the frontend's
// scratch. The host keeps a mirror of each stream's parity (it decides which
// streams step, so the mirror is exact) to tell callers where to upload.
#include <string.h>

#include <array>
#include <new>
#include <vector>

#include "detect_dev.cuh"
#include "frame.cuh"

namespace {

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct Group {
  vio_stream_group spec;
  vio_pyr_layout layout;
  int n_cells;
  uint8_t* frames;            // [2 slots][ns][2 cams] x h*w
  uint8_t* pyr;               // [2 slots][ns][2 cams] x upper_bytes
  float* list_xy;
  int32_t* list_id;
  int32_t* list_count;
  uint8_t* list_status;
  float* trk_xy;
  uint8_t* trk_status;
  unsigned long long* cand;
  int32_t* cand_count;
  float* spec_xy;
  uint8_t* spec_status;
  uint8_t* occupancy;
  float* new_xy;
  int32_t* new_count;
  int32_t* next_id;
  int32_t* stats;
  int32_t* step_ctr;
  int32_t* parity;
  int32_t* have_prev;
  int32_t* active;            // points into the batch's device mask
  float* net_out;             // flow proposals, [stream][camera] x cap x 3
  uint8_t* trk_learned;
  std::vector<int32_t> host_parity;
};

}  // namespace

struct vio_batch {
  std::vector<Group> groups;
  int total_streams;
  void* d_mem;
  int32_t* d_active;          // total_streams
  int32_t* h_active[2];       // pinned staging of the activity mask
  int mask_slot;
  vio::FrameTune tune;
  bool use_graph;
  cudaGraphExec_t graph[2];
  cudaEvent_t graph_done[2];
  bool graph_ready;
  const void* net;            // packed initializer weights (null: off)
  vio_initnet_cfg net_cfg;
};

namespace {

bool batch_params_ok(const vio_params* p) {
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

// Validates one group and lists the sizes of its device buffers.
vio_status group_sizes(const vio_stream_group& sp, vio_pyr_layout& layout, int& n_cells,
                       std::array<size_t, 26>& z) {
  if (!batch_params_ok(&sp.params) || sp.w < 1 || sp.h < 1 || sp.n_streams < 1 ||
      sp.capacity < 1 || sp.capacity > 32767)
    return VIO_ERR_INVALID_ARG;
  if (vio_pyr_layout_make(sp.w, sp.h, sp.params.n_levels, sp.w, &layout) != VIO_OK)
    return VIO_ERR_INVALID_ARG;
  const long long gx = sp.w / sp.params.cell_w, gy = sp.h / sp.params.cell_h;
  n_cells = (int)(gx * gy);
  if ((long long)n_cells * sp.params.k_per_cell > sp.capacity ||
      (long long)n_cells * 4 > 200 * 1024 ||
      !vio::det::detect_fits(sp.params.cell_w, sp.params.cell_h, sp.params.k_per_cell))
    return VIO_ERR_UNSUPPORTED;
  const size_t ns = sp.n_streams, cap = sp.capacity, nc = n_cells;
  const size_t kk = sp.params.k_per_cell, fb = (size_t)sp.w * sp.h;
  const size_t lists = 2 * ns * 2 * cap;
  z = {4 * ns * fb,                                  // frames
       4 * ns * (size_t)layout.upper_bytes,          // pyr
       lists * 8, lists * 4, 2 * ns * 2 * 4, lists,  // lists
       ns * 2 * cap * 8, ns * 2 * cap,               // trk
       ns * nc * kk * 8, ns * nc * 4,                // cand
       ns * nc * kk * 8, ns * nc * kk,               // spec
       ns * nc,                                      // occupancy
       ns * cap * 8, ns * 4, ns * 4,                 // new, next_id
       (size_t)VIO_STATS_RING * ns * VIO_N_STATS * 4,  // stats
       16, ns * 4, ns * 4,                           // step_ctr, parity, have_prev
       ns * 2 * cap * 12, ns * 2 * cap,              // net_out, trk_learned
       0, 0, 0, 0};
  return VIO_OK;
}

vio::FrameLaunch launch_of(Group& G) {
  using namespace vio;
  const vio_stream_group& sp = G.spec;
  const int ns = sp.n_streams;
  FrameLaunch f{};
  f.p = sp.params;
  f.g = make_geom(G.layout);
  f.n_streams = ns;
  f.cap = sp.capacity;
  const long long fb = (long long)sp.w * sp.h;
  f.cur = Batch{G.frames, fb, G.pyr, G.layout.upper_bytes, 4 * ns};
  f.prev = f.cur;
  f.slotted = 1;
  f.parity = G.parity;
  f.have_prev = G.have_prev;
  f.active = G.active;
  f.list_xy = G.list_xy;
  f.list_id = G.list_id;
  f.list_count = G.list_count;
  f.list_status = G.list_status;
  f.trk_xy = G.trk_xy;
  f.trk_status = G.trk_status;
  f.cand = G.cand;
  f.cand_count = G.cand_count;
  f.spec_xy = G.spec_xy;
  f.spec_status = G.spec_status;
  f.new_xy = G.new_xy;
  f.new_count = G.new_count;
  f.next_id = G.next_id;
  f.occupancy = G.occupancy;
  f.stats = G.stats;
  f.step_ctr = G.step_ctr;
  return f;
}

cudaError_t enqueue_step(vio_batch* b, const int32_t* h_mask, cudaStream_t s) {
  // activity mask: pinned staging -> device, then the launches
  cudaError_t e = cudaMemcpyAsync(b->d_active, h_mask, (size_t)b->total_streams * 4,
                                  cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return e;
  vio::FrameLaunch fl[vio::kMaxGroups];
  const int n = (int)b->groups.size();
  for (int i = 0; i < n; ++i) {
    fl[i] = launch_of(b->groups[i]);
    if (b->net) {
      fl[i].net = b->net;
      fl[i].net_la = b->net_cfg.level_a;
      fl[i].net_lb = b->net_cfg.level_b;
      fl[i].net_top = b->net_cfg.start_level;
      fl[i].net_tau = b->net_cfg.min_conf;
      fl[i].net_max_step = b->net_cfg.max_last_step;
      fl[i].net_out = b->groups[i].net_out;
      fl[i].trk_learned = b->groups[i].trk_learned;
    }
  }
  return vio::launch_frames(fl, n, b->tune, s, nullptr);
}

void mirror_parity(vio_batch* b, const int32_t* mask) {
  int k = 0;
  for (auto& G : b->groups)
    for (int s = 0; s < G.spec.n_streams; ++s, ++k)
      if (!mask || mask[k]) G.host_parity[s] ^= 1;
}

void drop_graphs(vio_batch* b) {
  if (b->graph_ready) {
    for (int i = 0; i < 2; ++i) cudaGraphExecDestroy(b->graph[i]);
    b->graph_ready = false;
  }
}

}  // namespace

extern "C" vio_status vio_batch_create(vio_batch** out, const vio_stream_group* groups,
                                       int32_t n_groups) {
  if (!out || !groups || n_groups < 1 || n_groups > vio::kMaxGroups) return VIO_ERR_INVALID_ARG;
  *out = nullptr;
  vio_batch* b = new (std::nothrow) vio_batch();
  if (!b) return VIO_ERR_OOM;
  b->groups.resize(n_groups);
  b->total_streams = 0;
  size_t total = 0;
  std::vector<std::array<size_t, 26>> sizes(n_groups);
  for (int i = 0; i < n_groups; ++i) {
    const vio_stream_group& sp = groups[i];
    Group& G = b->groups[i];
    G.spec = sp;
    const vio_status st = group_sizes(sp, G.layout, G.n_cells, sizes[i]);
    if (st != VIO_OK) {
      delete b;
      return st;
    }
    for (size_t v : sizes[i]) total += align256(v);
    b->total_streams += sp.n_streams;
  }
  total += align256((size_t)b->total_streams * 4);
  if (cudaMalloc(&b->d_mem, total) != cudaSuccess) {
    cudaGetLastError();
    delete b;
    return VIO_ERR_OOM;
  }
  if (cudaMallocHost(&b->h_active[0], (size_t)b->total_streams * 4) != cudaSuccess ||
      cudaMallocHost(&b->h_active[1], (size_t)b->total_streams * 4) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(b->d_mem);
    delete b;
    return VIO_ERR_OOM;
  }
  uint8_t* q = (uint8_t*)b->d_mem;
  auto take = [&](size_t n) {
    uint8_t* p = q;
    q += align256(n);
    return p;
  };
  int first = 0;
  b->d_active = nullptr;
  std::vector<uint8_t*> bases;
  for (int i = 0; i < n_groups; ++i) {
    Group& G = b->groups[i];
    auto& z = sizes[i];
    G.frames = take(z[0]);
    G.pyr = take(z[1]);
    G.list_xy = (float*)take(z[2]);
    G.list_id = (int32_t*)take(z[3]);
    G.list_count = (int32_t*)take(z[4]);
    G.list_status = take(z[5]);
    G.trk_xy = (float*)take(z[6]);
    G.trk_status = take(z[7]);
    G.cand = (unsigned long long*)take(z[8]);
    G.cand_count = (int32_t*)take(z[9]);
    G.spec_xy = (float*)take(z[10]);
    G.spec_status = take(z[11]);
    G.occupancy = take(z[12]);
    G.new_xy = (float*)take(z[13]);
    G.new_count = (int32_t*)take(z[14]);
    G.next_id = (int32_t*)take(z[15]);
    G.stats = (int32_t*)take(z[16]);
    G.step_ctr = (int32_t*)take(z[17]);
    G.parity = (int32_t*)take(z[18]);
    G.have_prev = (int32_t*)take(z[19]);
    G.net_out = (float*)take(z[20]);
    G.trk_learned = take(z[21]);
    G.host_parity.assign(G.spec.n_streams, 0);
  }
  b->d_active = (int32_t*)take((size_t)b->total_streams * 4);
  for (auto& G : b->groups) {
    G.active = b->d_active + first;
    first += G.spec.n_streams;
  }
  if (cudaMemset(b->d_mem, 0, total) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) {
    cudaGetLastError();
    cudaFreeHost(b->h_active[0]);
    cudaFreeHost(b->h_active[1]);
    cudaFree(b->d_mem);
    delete b;
    return VIO_ERR_CUDA;
  }
  for (auto& G : b->groups) {
    const size_t lists = 2 * (size_t)G.spec.n_streams * 2 * G.spec.capacity;
    cudaMemset(G.list_status, VIO_TRACK_EMPTY, lists);
  }
  b->mask_slot = 0;
  b->tune = vio::FrameTune{128, 0, 0, 0, 256};
  b->use_graph = false;
  b->graph_ready = false;
  b->graph_done[0] = b->graph_done[1] = nullptr;
  b->net = nullptr;
  b->net_cfg = vio_initnet_cfg{};
  if (cudaEventCreateWithFlags(&b->graph_done[0], cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->graph_done[1], cudaEventDisableTiming) != cudaSuccess ||
      cudaDeviceSynchronize() != cudaSuccess) {
    cudaGetLastError();
    vio_batch_destroy(b);
    return VIO_ERR_CUDA;
  }
  *out = b;
  return VIO_OK;
}

extern "C" vio_status vio_batch_destroy(vio_batch* b) {
  if (!b) return VIO_ERR_INVALID_ARG;
  drop_graphs(b);
  for (int i = 0; i < 2; ++i) {
    if (b->graph_done[i]) cudaEventDestroy(b->graph_done[i]);
    if (b->h_active[i]) cudaFreeHost(b->h_active[i]);
  }
  cudaFree(b->d_mem);
  delete b;
  return VIO_OK;
}

extern "C" vio_status vio_batch_next_frame(vio_batch* b, int32_t g, int32_t s,
                                           uint8_t** d_frame) {
  if (!b || !d_frame || g < 0 || g >= (int)b->groups.size()) return VIO_ERR_INVALID_ARG;
  Group& G = b->groups[g];
  if (s < 0 || s >= G.spec.n_streams) return VIO_ERR_INVALID_ARG;
  const size_t fb = (size_t)G.spec.w * G.spec.h;
  const int q = G.host_parity[s];
  *d_frame = G.frames + ((size_t)q * G.spec.n_streams + s) * 2 * fb;
  return VIO_OK;
}

extern "C" vio_status vio_batch_step(vio_batch* b, const int32_t* active, void* stream) {
  if (!b) return VIO_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const int slot = b->mask_slot;
  int32_t* hm = b->h_active[slot];
  bool same = true;   // an unchanged mask needs no rewrite, so no wait
  for (int i = 0; i < b->total_streams && same; ++i)
    same = hm[i] == (active ? (active[i] != 0) : 1);
  if (!same) {
    // the pinned buffer of this slot was last read by the step two calls ago
    if (cudaEventSynchronize(b->graph_done[slot]) != cudaSuccess) return VIO_ERR_CUDA;
    for (int i = 0; i < b->total_streams; ++i) hm[i] = active ? (active[i] != 0) : 1;
  }
  cudaError_t e;
  if (b->use_graph) {
    if (!s) return VIO_ERR_INVALID_ARG;   // the legacy default stream cannot be captured
    if (!b->graph_ready) {
      for (int i = 0; i < 2; ++i) {
        cudaGraph_t gr;
        e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return VIO_ERR_CUDA;
        const cudaError_t le = enqueue_step(b, b->h_active[i], s);
        e = cudaStreamEndCapture(s, &gr);
        if (le != cudaSuccess || e != cudaSuccess) return VIO_ERR_CUDA;
        e = cudaGraphInstantiate(&b->graph[i], gr, 0);
        cudaGraphDestroy(gr);
        if (e != cudaSuccess) return VIO_ERR_CUDA;
      }
      b->graph_ready = true;
    }
    e = cudaGraphLaunch(b->graph[slot], s);
  } else {
    e = enqueue_step(b, hm, s);
  }
  if (e != cudaSuccess) return VIO_ERR_CUDA;
  if (cudaEventRecord(b->graph_done[slot], s) != cudaSuccess) return VIO_ERR_CUDA;
  b->mask_slot ^= 1;
  mirror_parity(b, hm);
  return VIO_OK;
}

extern "C" vio_status vio_batch_set_graph(vio_batch* b, int32_t enable) {
  if (!b) return VIO_ERR_INVALID_ARG;
  b->use_graph = enable != 0;
  if (!b->use_graph) drop_graphs(b);
  return VIO_OK;
}

extern "C" vio_status vio_batch_set_tune(vio_batch* b, const vio_batch_tune* t) {
  if (!b || !t) return VIO_ERR_INVALID_ARG;
  if (t->k2_threads != 32 && t->k2_threads != 64 && t->k2_threads != 128 &&
      t->k2_threads != 256 && t->k2_threads != 512)
    return VIO_ERR_INVALID_ARG;
  if (t->pyr_tile_shift < -1 || t->pyr_tile_shift > 1) return VIO_ERR_INVALID_ARG;
  if (t->stereo_after_select != 0 && t->stereo_after_select != 1) return VIO_ERR_INVALID_ARG;
  if (t->pyr_first_levels < 0 || t->pyr_first_levels > 4) return VIO_ERR_INVALID_ARG;
  if (t->k1_threads != 128 && t->k1_threads != 256) return VIO_ERR_INVALID_ARG;
  if (t->det_warps != 0 && t->det_warps != 1 && t->det_warps != 2 && t->det_warps != 4 &&
      t->det_warps != 8)
    return VIO_ERR_INVALID_ARG;
  b->tune = vio::FrameTune{t->k2_threads, t->pyr_tile_shift, t->stereo_after_select,
                           t->pyr_first_levels, t->k1_threads, t->det_warps};
  drop_graphs(b);
  return VIO_OK;
}

extern "C" vio_status vio_batch_get_tune(vio_batch* b, vio_batch_tune* t) {
  if (!b || !t) return VIO_ERR_INVALID_ARG;
  t->k2_threads = b->tune.k2_threads;
  t->pyr_tile_shift = b->tune.pyr_tile_shift;
  t->stereo_after_select = b->tune.stereo_after;
  t->pyr_first_levels = b->tune.pyr_first;
  t->k1_threads = b->tune.k1_threads;
  t->det_warps = b->tune.det_warps;
  return VIO_OK;
}

extern "C" vio_status vio_batch_reset_stream(vio_batch* b, int32_t g, int32_t s, void* stream) {
  if (!b || g < 0 || g >= (int)b->groups.size()) return VIO_ERR_INVALID_ARG;
  Group& G = b->groups[g];
  if (s < 0 || s >= G.spec.n_streams) return VIO_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  cudaMemsetAsync(G.have_prev + s, 0, 4, st);
  cudaMemsetAsync(G.next_id + s, 0, 4, st);
  return cudaGetLastError() == cudaSuccess ? VIO_OK : VIO_ERR_CUDA;
}

namespace {
void reset_all(vio_batch* b, cudaStream_t st) {
  for (auto& G : b->groups) {
    cudaMemsetAsync(G.have_prev, 0, (size_t)G.spec.n_streams * 4, st);
    cudaMemsetAsync(G.next_id, 0, (size_t)G.spec.n_streams * 4, st);
    cudaMemsetAsync(G.parity, 0, (size_t)G.spec.n_streams * 4, st);
    G.host_parity.assign(G.spec.n_streams, 0);
  }
}
}  // namespace

extern "C" vio_status vio_batch_autotune(vio_batch* b, int32_t reps, void* stream,
                                         float* best_ms) {
  if (!b || reps < 1) return VIO_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const bool graph = b->use_graph;
  b->use_graph = false;
  drop_graphs(b);
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return VIO_ERR_CUDA;
  const int threads[5] = {32, 64, 128, 256, 512};
  float best = 1e30f;
  vio::FrameTune best_t = b->tune;
  vio_status st = VIO_OK;
  const int firsts[3] = {0, 2, 1};
  for (int combo = 0; combo < 180 && st == VIO_OK; ++combo) {
    const int ti = combo % 5, shift = (combo / 5) % 3 - 1, after = (combo / 15) % 2;
    const int first = firsts[(combo / 30) % 3], k1 = combo < 90 ? 256 : 128;
    {
      b->tune = vio::FrameTune{threads[ti], shift, after, first, k1, best_t.det_warps};
      float total = 0.f;
      for (int r = 0; r < reps; ++r) {
        reset_all(b, s);
        if (vio_batch_step(b, nullptr, s) != VIO_OK) {   // first frame: detection only
          st = VIO_ERR_CUDA;
          break;
        }
        cudaEventRecord(e0, s);
        if (vio_batch_step(b, nullptr, s) != VIO_OK) {   // tracked frame
          st = VIO_ERR_CUDA;
          break;
        }
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess) {
          st = VIO_ERR_CUDA;
          break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        total += ms;
      }
      if (st == VIO_OK && total / reps < best) {
        best = total / reps;
        best_t = b->tune;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  b->tune = best_t;
  reset_all(b, s);
  b->use_graph = graph;
  if (cudaStreamSynchronize(s) != cudaSuccess) st = VIO_ERR_CUDA;
  if (best_ms) *best_ms = best;
  return st;
}

extern "C" vio_status vio_batch_get_view(vio_batch* b, int32_t g, vio_frontend_view* out,
                                         int32_t* parity) {
  if (!b || !out || g < 0 || g >= (int)b->groups.size()) return VIO_ERR_INVALID_ARG;
  Group& G = b->groups[g];
  out->d_track_xy = G.list_xy;
  out->d_track_id = G.list_id;
  out->d_track_status = G.list_status;
  out->d_track_count = G.list_count;
  out->d_new_xy = G.new_xy;
  out->d_new_count = G.new_count;
  out->capacity = G.spec.capacity;
  out->n_streams = G.spec.n_streams;
  if (parity)
    for (int s = 0; s < G.spec.n_streams; ++s) parity[s] = G.host_parity[s];
  return VIO_OK;
}

extern "C" int32_t vio_batch_launches_per_step(const vio_batch* b) {
  if (!b) return 0;
  std::vector<vio::Geom> g;
  for (const auto& G : b->groups) g.push_back(vio::make_geom(G.layout));
  return vio::frame_launches(g.data(), (int)g.size(), b->net != nullptr,
                            b->tune.stereo_after != 0, b->tune.pyr_first);
}

extern "C" vio_status vio_batch_device_bytes(const vio_stream_group* groups, int32_t n_groups,
                                             int64_t* bytes) {
  if (!groups || !bytes || n_groups < 1 || n_groups > vio::kMaxGroups) return VIO_ERR_INVALID_ARG;
  int64_t total = 0, streams = 0;
  for (int i = 0; i < n_groups; ++i) {
    vio_pyr_layout L;
    int nc = 0;
    std::array<size_t, 26> z;
    const vio_status st = group_sizes(groups[i], L, nc, z);
    if (st != VIO_OK) return st;
    for (size_t v : z) total += (int64_t)align256(v);
    streams += groups[i].n_streams;
  }
  *bytes = total + (int64_t)align256((size_t)streams * 4);
  return VIO_OK;
}

extern "C" vio_status vio_batch_read_stats(vio_batch* b, int32_t g, int32_t* host_out,
                                           int64_t* n_steps) {
  if (!b || !host_out || !n_steps || g < 0 || g >= (int)b->groups.size())
    return VIO_ERR_INVALID_ARG;
  const Group& G = b->groups[g];
  const size_t bytes = (size_t)VIO_STATS_RING * G.spec.n_streams * VIO_N_STATS * 4;
  int32_t ctr = 0;
  if (cudaMemcpy(host_out, G.stats, bytes, cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(&ctr, G.step_ctr, 4, cudaMemcpyDeviceToHost) != cudaSuccess)
    return VIO_ERR_CUDA;
  *n_steps = ctr;
  return VIO_OK;
}

extern "C" vio_status vio_batch_set_initnet(vio_batch* b, const void* d_packed,
                                            const vio_initnet_cfg* cfg) {
  if (!b) return VIO_ERR_INVALID_ARG;
  if (d_packed) {
    for (const auto& G : b->groups)
      if (!vio::initnet_cfg_ok(cfg, G.spec.params.n_levels, d_packed))
        return VIO_ERR_INVALID_ARG;
    if (2 * b->total_streams > vio::KN_MAX_LISTS) return VIO_ERR_UNSUPPORTED;
    b->net_cfg = *cfg;
  }
  b->net = d_packed;
  drop_graphs(b);
  return VIO_OK;
}
