// The per-frame frontend as three dependent launches (Sec. III-B's stage
// order, with its data dependencies kept and its serialisation removed), for
// up to kMaxGroups groups of same-size stereo streams merged into each launch:
//
//  K1 frame_front_kernel    pyramid levels 1-4 of both cameras of every stream
//                           (one pyramid pass per tile) and, in the same
//                           launch, the per-cell FAST/NMS top-k candidates of
//                           camera 0. Levels beyond 4 follow as a further pass.
//  KN frame_initnet_kernel  (only with the learned initializer) persistent
//                           CTAs over rounds of 32 live tracks of one
//                           camera: network input from the previous and
//                           current pyramids, forward pass on the tcgen05
//                           tensor cores -> flow proposal + confidence.
//  K2 frame_track_kernel    one warp per keypoint: temporal tracking of every
//                           live track of both cameras (previous -> current
//                           pyramid; from the proposal over the lower levels
//                           when it is confident, the plain track otherwise
//                           or when that fails) AND stereo matching (camera 0
//                           -> 1) of every cell's top-k candidates.
//  K3 frame_finalize_kernel one CTA per stream: keep the tracks that passed,
//                           count them per cell, select per cell the first
//                           k - count candidates (the detection of Sec. III-D
//                           with the cell buffer), append them to camera 0 and
//                           their successful matches to camera 1.
//
// Matching every candidate, rather than only the selected ones, lets stereo
// matching run beside temporal tracking instead of after it. A keypoint's
// match depends only on its position and the two current pyramids, so the
// result for every selected keypoint is the one the sequential order gives;
// the candidates that the occupancy rejects are simply not used. That costs
// a match per cell per frame where only a few cells take new keypoints, so
// the other order is a tunable (stereo_after): K2 tracks temporally only,
// K3 selects and appends to camera 0, then
//  K4 frame_stereo_kernel   one warp per selected keypoint: stereo matching;
//  K5 frame_append_kernel   one CTA per stream: the successful matches, in
//                           order, appended to camera 1.
// Both orders give the same lists bit for bit.
//
// Streams are either stepped together with host-side parity (unslotted), or
// each keeps its own parity, first-frame flag and activity in device memory
// (slotted): inactive streams are skipped and keep their state, so one
// captured launch sequence serves any subset of streams.
#include "detect_dev.cuh"
#include "finalize_dev.cuh"
#include "frame.cuh"
#include "initnet_dev.cuh"
#include "initnet_tc.cuh"
#include "pyramid_dev.cuh"
#include "track_dev.cuh"

namespace vio {
namespace {


struct K1Args {
  Geom g;
  Batch all;           // images of the launch
  int m, T;            // levels and deepest-level tile of the first pyramid pass (m = 0: none)
  int ntx, nty;        // tiles of the first pass
  int det_step;        // 1: every image is a unit; 2: stream units (camera 0 detects)
  int blocks_per_unit; // det_step * tiles + detection blocks
  det::CellGeom cg;
  int n_cells, gy;
  const uint8_t* mask; // per detected image, or null
  long long mask_stride;
  unsigned long long* cand;
  int32_t* cand_count;
  int round_mode;
  // stream units (det_step == 2)
  int slotted, n_streams;
  const int32_t* parity;
  const int32_t* active;
  int32_t* step_ctr;   // incremented by block 0 (nullable)
  int32_t* ctr_copy;   // nullable: the new count is also stored here
};

struct MultiK1 {
  int n;
  long long block_end[kMaxGroups];
  K1Args a[kMaxGroups];
};

template <typename M>
__device__ __forceinline__ int group_of(const M& mm, long long i, long long& start) {
  int g = 0;
  while (g + 1 < mm.n && i >= mm.block_end[g]) ++g;
  start = g ? mm.block_end[g - 1] : 0;
  return g;
}

// Block layout per group: units, each unit = the pyramid tiles of its images
// followed by the detection cells of its first image, so that the blocks
// reading one image run together and its level 0 is read from DRAM about once.
// NT threads per CTA: 256 for a single frame's latency, 128 for throughput
// over many streams (a tunable of the batch).
template <int NT, bool MASKED>
__global__ void __launch_bounds__(NT, 768 / NT) frame_front_kernel(const __grid_constant__ MultiK1 mm) {
  extern __shared__ __align__(16) uint8_t smem[];
  long long start;
  const int gi = group_of(mm, blockIdx.x, start);
  const K1Args& a = mm.a[gi];
  const long long b = blockIdx.x - start;
  if (b == 0 && threadIdx.x == 0 && a.step_ctr) {
    const int c = *a.step_ctr + 1;
    *a.step_ctr = c;
    if (a.ctr_copy) *a.ctr_copy = c;
  }
  const int unit = (int)(b / a.blocks_per_unit);
  const int rem = (int)(b - (long long)unit * a.blocks_per_unit);
  int base = unit * a.det_step;
  if (a.det_step == 2 && a.slotted) {
    if (a.active && a.active[unit] == 0) return;
    base = 2 * (a.parity[unit] * a.n_streams + unit);
  }
  const int tiles = a.ntx * a.nty;
  const int n_pyr = a.m > 0 ? a.det_step * tiles : 0;
  if (rem < n_pyr) {
    const int img = base + rem / tiles;
    const int t = rem % tiles;
    const int ty = t / a.ntx, tx = t - ty * a.ntx;
    if (a.det_step == 2 || img < a.all.n)
      pyr::pyramid_pass(a.g, a.all, img, 0, a.m, a.T, tx, ty, a.ntx, a.nty, a.round_mode, smem);
    return;
  }
  det::detect_block<MASKED>(level_ptr(a.g, a.all, base, 0), a.g.w[0], a.g.h[0], a.g.pitch[0],
                            a.cg, a.gy, rem - n_pyr,
                            MASKED ? a.mask + (long long)unit * a.mask_stride : nullptr,
                            a.cand + (long long)unit * a.n_cells * a.cg.k,
                            a.cand_count + (long long)unit * a.n_cells, smem);
}

struct MultiK2 {
  int n;
  long long block_end[kMaxGroups];   // in warps here
  FrameLaunch f[kMaxGroups];
};

// Flow proposals of every live track: persistent CTAs over tiles of
// ntc::ROUND consecutive slots of one keypoint list (the temporal numbering of
// frame_track_kernel: list (2 stream + camera), slot); tiles past a list's
// count are skipped whole.
struct MultiKN {
  int n;
  long long block_end[kMaxGroups];   // in keypoint lists (2 per stream)
  int32_t* fault;                    // VIO_ERR_TIMEOUT when a completion wait gave up
  FrameLaunch f[kMaxGroups];
};

// Tile of the launch: a list's slots s0 .. s0 + nv - 1.
struct NetTile {
  int gi, list, s0, nv;
  StreamRef r;
  long long in_list;
};

static_assert(KN_MAX_LISTS * 4 + 64 + ntc::SMEM <= 227 * 1024,
              "shared memory of the proposal kernel");

// Per-list tile counts, prefix-summed in shared memory (every CTA), so that
// the tiles that hold keypoints are dealt out evenly over the CTAs.
struct NetLists {
  int n;                              // lists
  int* end;                           // inclusive prefix of tiles per list
};

__device__ __forceinline__ int list_tiles(const MultiKN& mm, int li, int& gi, int& list,
                                          long long& in_list, StreamRef& r) {
  long long start;
  gi = group_of(mm, li, start);       // block_end counts lists here
  const FrameLaunch& f = mm.f[gi];
  list = (int)(li - start);
  const int s = list >> 1, c = list & 1;
  r = stream_ref(f, s);
  if (!r.active || !r.have_prev) return 0;
  in_list = ((long long)r.li * f.n_streams + s) * 2 + c;
  const int count = min(f.list_count[in_list], f.cap);
  return (count + ntc::ROUND - 1) / ntc::ROUND;
}

__device__ __forceinline__ NetTile net_tile(const MultiKN& mm, const NetLists& L, int v) {
  // the list holding valid tile v: first prefix end above v
  int lo = 0, hi = L.n - 1;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (L.end[mid] > v) hi = mid; else lo = mid + 1;
  }
  NetTile T{};
  const int n_tiles = list_tiles(mm, lo, T.gi, T.list, T.in_list, T.r);
  const int j = v - (L.end[lo] - n_tiles);
  const FrameLaunch& f = mm.f[T.gi];
  const int count = min(f.list_count[T.in_list], f.cap);
  T.s0 = j * ntc::ROUND;
  T.nv = min(ntc::ROUND, count - T.s0);
  return T;
}

// Network inputs of a launch's tiles for ntc::run: the thread's row of a
// group, four channels (source / target at levels a and b) prefetched as
// aligned words.
struct KNSource {
  const MultiKN* mm;
  NetLists L;
  int n_valid;
  using Tile = NetTile;
  struct Regs {
    net::RowWords R[4];
    bool live;
  };
  __device__ int n_tiles() const { return n_valid; }
  __device__ Tile tile(int v) const { return net_tile(*mm, L, v); }
  __device__ void load(const Tile& T, int g, Regs& R) const {
    const FrameLaunch& f = mm->f[T.gi];
    const int i = g * ntc::GROUP + ntc::item_sample(), r = ntc::item_row(), c = T.list & 1;
    R.live = i < T.nv;
    if (!R.live) return;
    const float* xy = f.list_xy + 2 * (T.in_list * f.cap + T.s0 + i);
#pragma unroll
    for (int ch = 0; ch < 4; ++ch)
      net::row_prefetch(R.R[ch], f.g, (ch & 1) ? f.cur : f.prev,
                        ((ch & 1) ? T.r.cur_img : T.r.prev_img) + c,
                        ch < 2 ? f.net_la : f.net_lb, xy[0], xy[1], r);
  }
  __device__ void store(uint8_t* sm, const Regs& R) const {
    uint32_t px[4][4];
#pragma unroll
    for (int ch = 0; ch < 4; ++ch) {
      if (R.live) {
        ntc::row_bytes(R.R[ch], px[ch]);
      } else {
#pragma unroll
        for (int k = 0; k < 4; ++k) px[ch][k] = 0x80808080u;
      }
    }
    if (ntc::NH == 1 || (threadIdx.x >> 7))
      ntc::store_row_bytes<1>(sm, ntc::item_sample(), ntc::item_row(), px);
    if (ntc::NH == 1 || !(threadIdx.x >> 7))
      ntc::store_row_bytes<0>(sm, ntc::item_sample(), ntc::item_row(), px);
  }
  __device__ void write(const Tile& T, int s, float dx, float dy, float conf) const {
    const FrameLaunch& f = mm->f[T.gi];
    float* o = f.net_out + 3 * ((long long)T.list * f.cap + T.s0 + s);
    o[0] = dx;
    o[1] = dy;
    o[2] = conf;
  }
};

// Persistent CTAs over the tiles that hold keypoints (valid tile v goes to
// CTA v mod gridDim.x). Needs level_a, level_b >= 1 (aligned level rows).
__global__ void __launch_bounds__(ntc::THREADS, 1) frame_initnet_kernel(
    const __grid_constant__ MultiKN mm) {
  extern __shared__ __align__(16) uint8_t sm[];
  __shared__ int ends[KN_MAX_LISTS];
  __shared__ int warp_tot[ntc::THREADS / 32];
  const int n_lists = (int)mm.block_end[mm.n - 1];
  // per-list tile counts and their inclusive prefix (chunks of blockDim.x)
  int carry = 0;
  for (int base = 0; base < n_lists; base += blockDim.x) {
    const int li = base + threadIdx.x;
    int nt = 0;
    if (li < n_lists) {
      int gi, list;
      long long in_list;
      StreamRef r;
      nt = list_tiles(mm, li, gi, list, in_list, r);
    }
    int incl = nt;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    int before = carry;
    for (int w = 0; w < warp; ++w) before += warp_tot[w];
    if (li < n_lists) ends[li] = before + incl;
    int tot = 0;
    for (int w = 0; w < ntc::THREADS / 32; ++w) tot += warp_tot[w];
    carry += tot;
    __syncthreads();
  }
  const KNSource src{&mm, NetLists{n_lists, ends}, carry};
  ntc::run(src, mm.f[0].net, sm, mm.fault);
}

// Occupancy hint of the tracking launch (blocks of up to 512 threads, this
// many per SM: 2 caps registers at 64 per thread); unset = compiler's choice.
#ifdef VIO_TRACK_MIN_BLOCKS
#define VIO_TRACK_BOUNDS __launch_bounds__(512, VIO_TRACK_MIN_BLOCKS)
#else
#define VIO_TRACK_BOUNDS
#endif

// BUTTERFLY: the reduction form for a launch that leaves most of the GPU
// idle (trk::warp_sum4).
template <bool BUTTERFLY>
__global__ void VIO_TRACK_BOUNDS frame_track_kernel(const __grid_constant__ MultiK2 mm) {
  // the finalisation (launched as this launch's programmatic dependent) may
  // take its SM now and wait there for this launch's completion
  asm volatile("griddepcontrol.launch_dependents;");
  const long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= mm.block_end[mm.n - 1]) return;
  long long start;
  const int gi = group_of(mm, w, start);
  const FrameLaunch& f = mm.f[gi];
  const long long wl = w - start;
  const float qnan = __int_as_float(0x7fc00000);
  const TrackCfg cfg{f.p.gn_iters, 1, f.p.fb_max_dist, -1};
  const int top = f.g.n_levels - 1;
  const long long n_temporal = 2LL * f.n_streams * f.cap;
  trk::Pos tf;
  float thf, dist;
  bool have;
  if (wl < n_temporal) {
    const int list = (int)(wl / f.cap);       // 2s + c
    const int slot = (int)(wl - (long long)list * f.cap);
    const int s = list >> 1, c = list & 1;
    const StreamRef r = stream_ref(f, s);
    if (!r.active) return;
    const long long in_list = ((long long)r.li * f.n_streams + s) * 2 + c;
    if (!r.have_prev || slot >= f.list_count[in_list]) {
      if (lane == 0) f.trk_status[wl] = VIO_TRACK_EMPTY;
      return;
    }
    const long long src = in_list * f.cap + slot;
    const float px = f.list_xy[2 * src], py = f.list_xy[2 * src + 1];
    int st = VIO_TRACK_EMPTY;
    bool learned = false;
    if (f.net) {
      const float* q = f.net_out + 3 * wl;
      if (q[2] >= f.net_tau) {
        float last;
        st = trk::track_fb<BUTTERFLY>(f.g, f.prev, r.prev_img + c, f.cur, r.cur_img + c, px, py,
                                      true, px + q[0], py + q[1], 0.f, cfg, f.net_top, lane, tf,
                                      thf, have, dist, last);
        learned = st == VIO_TRACK_OK && !(f.net_max_step > 0.f && last > f.net_max_step);
      }
    }
    if (!learned) {
      float last;
      st = trk::track_fb<BUTTERFLY>(f.g, f.prev, r.prev_img + c, f.cur, r.cur_img + c, px, py,
                                    false, 0.f, 0.f, 0.f, cfg, top, lane, tf, thf, have, dist,
                                    last);
    }
    if (lane == 0) {
      if (f.net) f.trk_learned[wl] = learned ? 1 : 0;
      f.trk_status[wl] = (uint8_t)st;
      f.trk_xy[2 * wl] = have ? (float)tf.ax + tf.dx : qnan;
      f.trk_xy[2 * wl + 1] = have ? (float)tf.ay + tf.dy : qnan;
    }
    return;
  }
  const long long w2 = wl - n_temporal;
  const int k = f.p.k_per_cell;
  const int n_cells = (f.g.w[0] / f.p.cell_w) * (f.g.h[0] / f.p.cell_h);
  const int per = n_cells * k;
  const int s = (int)(w2 / per);
  const int rem = (int)(w2 - (long long)s * per);
  const int cell = rem / k, rr = rem - cell * k;
  const StreamRef r = stream_ref(f, s);
  if (!r.active) return;
  if (rr >= f.cand_count[(long long)s * n_cells + cell]) {
    if (lane == 0) f.spec_status[w2] = VIO_TRACK_EMPTY;
    return;
  }
  const unsigned long long key = f.cand[w2];
  const unsigned idx = ~(unsigned)(key & 0xffffffffu);
  const float x = (float)(idx % (unsigned)f.g.w[0]), y = (float)(idx / (unsigned)f.g.w[0]);
  float last;
  const int st = trk::track_fb<BUTTERFLY>(f.g, f.cur, r.cur_img, f.cur, r.cur_img + 1, x, y,
                                          false, 0.f, 0.f, 0.f, cfg, top, lane, tf, thf, have,
                                          dist, last);
  if (lane == 0) {
    f.spec_status[w2] = (uint8_t)st;
    f.spec_xy[2 * w2] = have ? (float)tf.ax + tf.dx : qnan;
    f.spec_xy[2 * w2 + 1] = have ? (float)tf.ay + tf.dy : qnan;
  }
}

// Launches `kernel` on stream s, as a programmatic dependent of the previous
// launch when `dependent`: its CTAs may then be scheduled once every CTA of
// the previous launch has passed griddepcontrol.launch_dependents (or
// exited), and the kernel itself waits on griddepcontrol.wait before touching
// memory. Only after a launch that leaves most of the GPU idle (at most
// kDependentMaxWarpsPerSm warps per SM): after one that fills the GPU, the
// dependent's early-resident CTAs (a 1024-thread CTA holds all of an SM's
// registers) would slow it more than the launch latency they hide.
constexpr int kDependentMaxWarpsPerSm = 16;
template <class K, class A>
cudaError_t launch_dependent(K kernel, unsigned grid, unsigned block, size_t smem,
                             cudaStream_t s, const A& args, bool dependent = true) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = dependent ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kernel, args);
}

struct MultiK3 {
  int n;
  long long block_end[kMaxGroups];   // in blocks (= streams)
  FrameLaunch f[kMaxGroups];
};

// One CTA per stream. Each thread owns a contiguous run of list slots (then
// of cells), so each phase is one block-wide scan of packed counts.
__global__ void __launch_bounds__(K3_THREADS)
    frame_finalize_kernel(const __grid_constant__ MultiK3 mm) {
  // launched as the tracking launch's programmatic dependent: wait for its
  // completion and memory (a no-op after an ordinary launch); the stereo
  // launch that may follow can be scheduled now
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;");
  extern __shared__ int occ_s[];
  __shared__ int ws32[K3_THREADS / 32];
  __shared__ unsigned long long ws64[K3_THREADS / 32];
  long long start;
  const int gi = group_of(mm, blockIdx.x, start);
  const FrameLaunch& f = mm.f[gi];
  const int s = (int)(blockIdx.x - start);
  finalize_stream(f, s, occ_s, ws32, ws64);
}

// ---- the after-selection order: stereo matching of the selected keypoints

// Selected keypoints a stream can have: every cell's k, at most the capacity.
__host__ __device__ inline int max_new(const FrameLaunch& f) {
  const int n = (f.g.w[0] / f.p.cell_w) * (f.g.h[0] / f.p.cell_h) * f.p.k_per_cell;
  return n < f.cap ? n : f.cap;
}

__global__ void frame_stereo_kernel(const __grid_constant__ MultiK2 mm) {
  // a programmatic dependent of the finalisation; the append may be
  // scheduled now
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;");
  const long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= mm.block_end[mm.n - 1]) return;
  long long start;
  const int gi = group_of(mm, w, start);
  const FrameLaunch& f = mm.f[gi];
  const int mn = max_new(f);
  const long long wl = w - start;
  const int s = (int)(wl / mn), slot = (int)(wl - (long long)s * mn);
  const StreamRef r = stream_ref(f, s);
  if (!r.active || slot >= f.new_count[s]) return;
  const long long q = (long long)s * f.cap + slot;
  const TrackCfg cfg{f.p.gn_iters, 1, f.p.fb_max_dist, -1};
  trk::Pos tf;
  float thf, dist, last;
  bool have;
  const int st = trk::track_fb(f.g, f.cur, r.cur_img, f.cur, r.cur_img + 1, f.new_xy[2 * q],
                               f.new_xy[2 * q + 1], false, 0.f, 0.f, 0.f, cfg,
                               f.g.n_levels - 1, lane, tf, thf, have, dist, last);
  if (lane == 0) {
    const long long o = (long long)s * mn + slot;
    f.spec_status[o] = (uint8_t)st;
    f.spec_xy[2 * o] = have ? (float)tf.ax + tf.dx : __int_as_float(0x7fc00000);
    f.spec_xy[2 * o + 1] = have ? (float)tf.ay + tf.dy : __int_as_float(0x7fc00000);
  }
}

// Appends the successful matches of a stream's selected keypoints, in their
// order, to camera 1 after its surviving tracks, and ends the stream's step.
__global__ void __launch_bounds__(K3_THREADS)
    frame_append_kernel(const __grid_constant__ MultiK3 mm) {
  asm volatile("griddepcontrol.wait;" ::: "memory");   // after the stereo matching
  __shared__ int ws32[K3_THREADS / 32];
  long long start;
  const int gi = group_of(mm, blockIdx.x, start);
  const FrameLaunch& f = mm.f[gi];
  const int s = (int)(blockIdx.x - start);
  const StreamRef sr = stream_ref(f, s);
  if (!sr.active) return;
  const int t = threadIdx.x;
  const long long cap = f.cap;
  const int mn = max_new(f);
  const long long cnt_out = ((long long)sr.lo * f.n_streams + s) * 2;
  const long long out1 = (cnt_out + 1) * cap;
  const int surv1 = f.list_count[cnt_out + 1];           // K3 left the survivors' count
  const int ctr = *(f.ctr_copy ? f.ctr_copy : f.step_ctr);
  int32_t* st = f.stats + ((long long)((ctr - 1) % VIO_STATS_RING) * f.n_streams + s) * VIO_N_STATS;
  const int n_new = f.new_count[s];
  const int id0 = f.next_id[s] - st[VIO_STAT_NEW];
  const int run = (n_new + K3_THREADS - 1) / K3_THREADS;
  int m_tot = 0;
  for (int r0 = 0; r0 < run; r0 += kRunMax) {
    const int rl = min(kRunMax, run - r0);
    const int first = t * run + r0;
    unsigned keep = 0;
    for (int j = 0; j < rl; ++j) {
      const int i = first + j;
      if (i < n_new && f.spec_status[(long long)s * mn + i] == VIO_TRACK_OK) keep |= 1u << j;
    }
    int tot;
    int o = m_tot + block_scan<int>(__popc(keep), ws32, tot);
    for (int j = 0; j < rl; ++j) {
      if (!(keep & (1u << j))) continue;
      const int i = first + j;
      const int o1 = surv1 + o++;
      if (o1 < f.cap) {
        const long long q = (long long)s * mn + i;
        f.list_xy[2 * (out1 + o1)] = f.spec_xy[2 * q];
        f.list_xy[2 * (out1 + o1) + 1] = f.spec_xy[2 * q + 1];
        f.list_id[out1 + o1] = id0 + i;
        f.list_status[out1 + o1] = VIO_TRACK_OK;
      }
    }
    m_tot += tot;
    __syncthreads();
  }
  if (t == 0) {
    f.list_count[cnt_out + 1] = min(surv1 + m_tot, f.cap);
    st[VIO_STAT_MATCHED] = m_tot;
    if (f.slotted) {
      f.parity[s] = sr.lo;
      f.have_prev[s] = 1;
    }
  }
}

// Levels the fused pass of K1 computes (the rest follow in further passes).
int first_levels(const Geom& g, int pyr_first) {
  const int m = g.n_levels > 1 ? pyr::pass_levels(g.n_levels, 0) : 0;
  return (pyr_first > 0 && pyr_first < m) ? pyr_first : m;
}

K1Args front_args(const vio_params& p, const Geom& g, const Batch& all, int det_step,
                  const uint8_t* mask, long long mask_stride, unsigned long long* cand,
                  int32_t* cand_count, int tile_shift, int pyr_first, int threads,
                  int det_warps) {
  const int gx = g.w[0] / p.cell_w, gy = g.h[0] / p.cell_h;
  K1Args a{};
  a.g = g;
  a.all = all;
  a.m = first_levels(g, pyr_first);
  a.T = a.m > 0 ? pyr::top_tile(a.m, tile_shift) : 1;
  a.ntx = a.nty = 1;
  if (a.m > 0) pyr::pass_tiles(g.w, g.h, 0, a.m, a.T, a.ntx, a.nty);
  a.det_step = det_step;
  a.n_cells = gx * gy;
  a.gy = gy;
  a.cg = det::CellGeom{p.cell_w, p.cell_h, gx, p.k_per_cell, p.thresholds[p.n_thresholds - 1],
                       p.detect_border, 1, 1, 1, p.select_mode};
  det::detect_setup(a.cg, threads, det_warps);
  a.blocks_per_unit = (a.m > 0 ? det_step * a.ntx * a.nty : 0) +
                      (a.n_cells > 0 ? det::detect_blocks(gx, gy, a.cg.bcx, a.cg.bcy) : 0);
  a.mask = mask;
  a.mask_stride = mask_stride;
  a.cand = cand;
  a.cand_count = cand_count;
  a.round_mode = p.round_mode;
  return a;
}

template <int NT, bool MASKED>
cudaError_t launch_k1_nt(const MultiK1& mm, int smem, cudaStream_t s) {
  if (smem > 48 * 1024) {
    const cudaError_t e = cudaFuncSetAttribute(
        frame_front_kernel<NT, MASKED>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
  }
  const long long blocks = mm.block_end[mm.n - 1];
  if (blocks > 0) frame_front_kernel<NT, MASKED><<<(unsigned)blocks, NT, smem, s>>>(mm);
  return cudaGetLastError();
}

// MASKED when any group of the launch has a per-pixel detection mask.
cudaError_t launch_k1(const MultiK1& mm, int smem, int threads, cudaStream_t s) {
  bool masked = false;
  for (int i = 0; i < mm.n; ++i) masked = masked || mm.a[i].mask != nullptr;
  if (masked)
    return threads == 128 ? launch_k1_nt<128, true>(mm, smem, s)
                          : launch_k1_nt<256, true>(mm, smem, s);
  return threads == 128 ? launch_k1_nt<128, false>(mm, smem, s)
                        : launch_k1_nt<256, false>(mm, smem, s);
}

}  // namespace

int frame_front_smem(const Geom& g, const vio_params& p, int tile_shift, int pyr_first,
                     int threads, int det_warps) {
  det::CellGeom cg{p.cell_w, p.cell_h, g.w[0] / p.cell_w, p.k_per_cell, 0, 0, 1, 1, 1};
  int smem = det::detect_setup(cg, threads, det_warps);
  const int m = first_levels(g, pyr_first);
  if (m > 0) {
    const int ps = pyr::pass_smem_max(g.w, g.h, 0, m, pyr::top_tile(m, tile_shift));
    smem = ps > smem ? ps : smem;
  }
  return smem;
}

cudaError_t launch_frames(const FrameLaunch* fl, int n_groups, const FrameTune& tune,
                          cudaStream_t s, cudaEvent_t* marks, int part) {
  if (n_groups < 1 || n_groups > kMaxGroups) return cudaErrorInvalidValue;
  auto mark = [&](int i) {
    if (marks && marks[i]) cudaEventRecord(marks[i], s);
  };

  cudaError_t e = cudaSuccess;
  long long acc = 0;
  if (part != 2) {
    // K1: pyramid levels 1-4 + detection candidates (camera 0 of each stream)
    mark(0);
    MultiK1 m1{};
    m1.n = n_groups;
    int smem1 = 0;
    long long cells = 0;
    for (int i = 0; i < n_groups; ++i)
      cells += (long long)fl[i].n_streams * (fl[i].g.w[0] / fl[i].p.cell_w) *
               (fl[i].g.h[0] / fl[i].p.cell_h);
    const int gw = tune.det_warps > 0 ? tune.det_warps : det::warps_per_cell(cells, sm_count());
    for (int i = 0; i < n_groups; ++i) {
      const FrameLaunch& f = fl[i];
      K1Args a = front_args(f.p, f.g, f.cur, 2, nullptr, 0, f.cand, f.cand_count,
                            tune.pyr_tile_shift, tune.pyr_first, tune.k1_threads, gw);
      a.slotted = f.slotted;
      a.n_streams = f.n_streams;
      a.parity = f.parity;
      a.active = f.active;
      a.step_ctr = f.step_ctr;
      a.ctr_copy = f.ctr_copy;
      m1.a[i] = a;
      acc += (long long)f.n_streams * a.blocks_per_unit;
      m1.block_end[i] = acc;
      const int sm = frame_front_smem(f.g, f.p, tune.pyr_tile_shift, tune.pyr_first,
                                      tune.k1_threads, gw);
      smem1 = sm > smem1 ? sm : smem1;
    }
    e = launch_k1(m1, smem1, tune.k1_threads, s);
    if (e != cudaSuccess) return e;
    // levels beyond the first pass
    mark(1);
    for (int i = 0; i < n_groups; ++i) {
      const FrameLaunch& f = fl[i];
      const int m1 = first_levels(f.g, tune.pyr_first);
      if (f.g.n_levels > 1 + m1) {
        e = launch_pyramid_from(f.g, f.cur, m1, f.p.round_mode, s);
        if (e != cudaSuccess) return e;
      }
    }
  }
  if (part == 1) return cudaGetLastError();

  // KN: flow proposals (every group has the initializer on, or none)
  mark(2);
  if (fl[0].net) {
    MultiKN mn{};
    mn.n = n_groups;
    acc = 0;                                    // keypoint lists
    long long tiles = 0;                        // tiles if every list were full
    for (int i = 0; i < n_groups; ++i) {
      mn.f[i] = fl[i];
      acc += 2LL * fl[i].n_streams;
      tiles += 2LL * fl[i].n_streams * ((fl[i].cap + ntc::ROUND - 1) / ntc::ROUND);
      mn.block_end[i] = acc;
    }
    if (acc > KN_MAX_LISTS) return cudaErrorInvalidValue;
    static PerDeviceOnce kn_attr;
    e = once_per_device(kn_attr, [] {
      return cudaFuncSetAttribute(frame_initnet_kernel,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, ntc::SMEM);
    });
    if (e != cudaSuccess) return e;
    mn.fault = net_fault_word();
    const int sms = sm_count();
    const long long blocks = tiles < sms ? tiles : sms;
    if (blocks > 0)
      frame_initnet_kernel<<<(unsigned)blocks, ntc::THREADS, ntc::SMEM, s>>>(mn);
  }

  // K2: temporal tracking + stereo matching of all candidates
  mark(3);
  MultiK2 m2{};
  m2.n = n_groups;
  acc = 0;
  for (int i = 0; i < n_groups; ++i) {
    const FrameLaunch& f = fl[i];
    m2.f[i] = f;
    m2.f[i].stereo_after = tune.stereo_after;
    const int n_cells = (f.g.w[0] / f.p.cell_w) * (f.g.h[0] / f.p.cell_h);
    acc += 2LL * f.n_streams * f.cap +
           (tune.stereo_after ? 0LL : (long long)f.n_streams * n_cells * f.p.k_per_cell);
    m2.block_end[i] = acc;
  }
  const int k2t = tune.k2_threads;
  const bool k2_small = acc <= (long long)kDependentMaxWarpsPerSm * sm_count();
  if (acc > 0) {
    const long long blocks2 = (acc * 32 + k2t - 1) / k2t;
    if (k2_small)
      frame_track_kernel<true><<<(unsigned)blocks2, k2t, 0, s>>>(m2);
    else
      frame_track_kernel<false><<<(unsigned)blocks2, k2t, 0, s>>>(m2);
  }

  // K3: finalize
  mark(4);
  MultiK3 m3{};
  m3.n = n_groups;
  acc = 0;
  int smem3 = 0;
  for (int i = 0; i < n_groups; ++i) {
    const FrameLaunch& f = fl[i];
    m3.f[i] = f;
    m3.f[i].stereo_after = tune.stereo_after;
    acc += f.n_streams;
    m3.block_end[i] = acc;
    const int sm = (f.g.w[0] / f.p.cell_w) * (f.g.h[0] / f.p.cell_h) * (int)sizeof(int);
    smem3 = sm > smem3 ? sm : smem3;
  }
  if (smem3 > 48 * 1024) {
    e = cudaFuncSetAttribute(frame_finalize_kernel,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, smem3);
    if (e != cudaSuccess) return e;
  }
  // a programmatic dependent of a small tracking launch (a single frame): its
  // CTA is resident and waiting when the tracking ends
  e = launch_dependent(frame_finalize_kernel, (unsigned)acc, K3_THREADS, (size_t)smem3, s, m3,
                       k2_small);
  if (e != cudaSuccess) return e;
  if (tune.stereo_after) {
    // K4: stereo matching of the selected keypoints; K5: append to camera 1
    MultiK2 m4{};
    m4.n = n_groups;
    long long w4 = 0;
    for (int i = 0; i < n_groups; ++i) {
      m4.f[i] = m3.f[i];
      w4 += (long long)fl[i].n_streams * max_new(fl[i]);
      m4.block_end[i] = w4;
    }
    if (w4 > 0) {
      const long long blocks4 = (w4 * 32 + k2t - 1) / k2t;
      e = launch_dependent(frame_stereo_kernel, (unsigned)blocks4, (unsigned)k2t, 0, s, m4);
      if (e != cudaSuccess) return e;
    }
    e = launch_dependent(frame_append_kernel, (unsigned)acc, K3_THREADS, 0, s, m3,
                         w4 <= (long long)kDependentMaxWarpsPerSm * sm_count());
    if (e != cudaSuccess) return e;
  }
  mark(5);
  return cudaGetLastError();
}

int frame_launches(const Geom* g, int n_groups, bool with_net, bool stereo_after,
                   int pyr_first) {
  int n = (with_net ? 4 : 3) + (stereo_after ? 2 : 0);   // K1, (KN), K2, K3, (K4, K5)
  for (int i = 0; i < n_groups; ++i) {
    const int rest = g[i].n_levels - 1 - first_levels(g[i], pyr_first);
    if (rest > 0) n += pyr::rest_passes(rest);
  }
  return n;
}

}  // namespace vio
