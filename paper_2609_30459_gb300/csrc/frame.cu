// The per-frame frontend as three dependent launches (Sec. III-B's stage
// order, with its data dependencies kept and its serialisation removed):
//
//  K1 frame_front_kernel   pyramid levels 1-4 of every image (one pyramid
//                          pass per tile) and, in the same launch, the
//                          per-cell FAST/NMS top-k candidates of camera 0.
//                          Levels beyond 4 follow as a further pass.
//  K2 frame_track_kernel   one warp per keypoint: temporal tracking of every
//                          live track of both cameras (previous -> current
//                          pyramid) AND stereo matching (camera 0 -> 1) of
//                          every cell's top-k candidates.
//  K3 frame_finalize_kernel one CTA per stream: keep the tracks that passed,
//                          count them per cell, select per cell the first
//                          k - count candidates (the detection of Sec. III-D
//                          with the cell buffer), append them to camera 0 and
//                          their successful matches to camera 1.
//
// Matching every candidate, rather than only the selected ones, lets stereo
// matching run beside temporal tracking instead of after it. A keypoint's
// match depends only on its position and the two current pyramids, so the
// result for every selected keypoint is the one the sequential order gives;
// the candidates that the occupancy rejects are simply not used.
#include "detect_dev.cuh"
#include "frame.cuh"
#include "pyramid_dev.cuh"
#include "track_dev.cuh"

namespace vio {
namespace {

constexpr int K1_THREADS = 256;
static_assert(K1_THREADS == pyr::kThreads && K1_THREADS == det::kThreads, "block size");

struct K1Args {
  Geom g;
  Batch all;           // every image of the batch
  int m;               // levels of the first pass (1..4; 0 = no pyramid)
  int ntx, nty;        // tiles of the first pass
  int det_step;        // detection on every det_step-th image (1 or 2)
  int blocks_per_unit; // det_step * tiles + cells
  det::CellGeom cg;
  int n_cells;
  const uint8_t* mask; // per detected image, or null
  long long mask_stride;
  unsigned long long* cand;
  int32_t* cand_count;
  int round_mode;
};

// Block layout: units of det_step images, each unit = the pyramid tiles of
// its images followed by the detection cells of its first image, so that the
// blocks reading one image run together and its level 0 is read from DRAM
// about once.
__global__ void __launch_bounds__(K1_THREADS) frame_front_kernel(K1Args a) {
  extern __shared__ __align__(16) uint8_t smem[];
  __shared__ unsigned long long red[K1_THREADS / 32];
  const int unit = blockIdx.x / a.blocks_per_unit;
  const int rem = blockIdx.x - unit * a.blocks_per_unit;
  const int tiles = a.ntx * a.nty;
  const int n_pyr = a.m > 0 ? a.det_step * tiles : 0;
  if (rem < n_pyr) {
    const int img = unit * a.det_step + rem / tiles;
    const int t = rem % tiles;
    const int ty = t / a.ntx, tx = t - ty * a.ntx;
    if (img < a.all.n)
      pyr::pyramid_pass(a.g, a.all, img, 0, a.m, tx, ty, a.ntx, a.nty, a.round_mode, smem);
    return;
  }
  const int cell = rem - n_pyr;
  const int img = unit * a.det_step;
  const long long slot = (long long)unit * a.n_cells + cell;
  det::detect_cell(level_ptr(a.g, a.all, img, 0), a.g.w[0], a.g.h[0], a.g.pitch[0], a.cg, cell,
                   a.mask ? a.mask + (long long)unit * a.mask_stride : nullptr,
                   a.cand + slot * a.cg.k, a.cand_count + slot, smem, red);
}

struct K2Args {
  Geom g;
  Batch prev, cur;
  const float* list_xy;
  const int32_t* list_count;
  int cap;
  long long n_temporal;     // warps of temporal work (0 on the first frame)
  float* trk_xy;
  uint8_t* trk_status;
  const unsigned long long* cand;
  const int32_t* cand_count;
  int n_cells, k, W;
  long long n_stereo;       // warps of stereo work
  float* spec_xy;
  uint8_t* spec_status;
  TrackCfg cfg;
};

constexpr int K2_THREADS = 128;

__global__ void __launch_bounds__(K2_THREADS) frame_track_kernel(K2Args a) {
  const long long w = ((long long)blockIdx.x * K2_THREADS + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const float qnan = __int_as_float(0x7fc00000);
  trk::Pos tf;
  float thf, dist;
  bool have;
  if (w < a.n_temporal) {
    const int list = (int)(w / a.cap);
    const int slot = (int)(w - (long long)list * a.cap);
    if (slot >= a.list_count[list]) {
      if (lane == 0) a.trk_status[w] = VIO_TRACK_EMPTY;
      return;
    }
    const int st = trk::track_fb(a.g, a.prev, list, a.cur, list, a.list_xy[2 * w],
                                 a.list_xy[2 * w + 1], nullptr, a.cfg, lane, tf, thf, have, dist);
    if (lane == 0) {
      a.trk_status[w] = (uint8_t)st;
      a.trk_xy[2 * w] = have ? (float)tf.ax + tf.dx : qnan;
      a.trk_xy[2 * w + 1] = have ? (float)tf.ay + tf.dy : qnan;
    }
    return;
  }
  const long long w2 = w - a.n_temporal;
  if (w2 >= a.n_stereo) return;
  const int per = a.n_cells * a.k;
  const int stream = (int)(w2 / per);
  const int rem = (int)(w2 - (long long)stream * per);
  const int cell = rem / a.k, r = rem - cell * a.k;
  if (r >= a.cand_count[(long long)stream * a.n_cells + cell]) {
    if (lane == 0) a.spec_status[w2] = VIO_TRACK_EMPTY;
    return;
  }
  const unsigned long long key = a.cand[w2];
  const unsigned idx = ~(unsigned)(key & 0xffffffffu);
  const float x = (float)(idx % (unsigned)a.W), y = (float)(idx / (unsigned)a.W);
  const int st = trk::track_fb(a.g, a.cur, 2 * stream, a.cur, 2 * stream + 1, x, y, nullptr,
                               a.cfg, lane, tf, thf, have, dist);
  if (lane == 0) {
    a.spec_status[w2] = (uint8_t)st;
    a.spec_xy[2 * w2] = have ? (float)tf.ax + tf.dx : qnan;
    a.spec_xy[2 * w2 + 1] = have ? (float)tf.ay + tf.dy : qnan;
  }
}

constexpr int K3_THREADS = 512;

// Block-wide exclusive scan (one value per thread); returns the exclusive
// prefix and the block total. All threads must call it.
template <typename T>
__device__ __forceinline__ T block_scan(T v, T* warp_sums, T& total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const T t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) warp_sums[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    T ws = lane < K3_THREADS / 32 ? warp_sums[lane] : T(0);
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const T t = __shfl_up_sync(0xffffffffu, ws, o);
      if (lane >= o) ws += t;
    }
    if (lane < K3_THREADS / 32) warp_sums[lane] = ws;
  }
  __syncthreads();
  total = warp_sums[K3_THREADS / 32 - 1];
  return (warp ? warp_sums[warp - 1] : T(0)) + incl - v;
}

__device__ __forceinline__ int cell_of(float x, int cw) {
  int c = (int)floorf(x / (float)cw);
  if ((float)(c + 1) * (float)cw <= x) ++c;
  if ((float)c * (float)cw > x) --c;
  return c;
}

struct K3Args {
  int have_prev, cap, k, W, gx, gy, cw, ch;
  // temporal results and the lists they came from
  const float* trk_xy;
  const uint8_t* trk_status;
  const int32_t* ids_in;
  const int32_t* count_in;
  // candidates and their matches
  const unsigned long long* cand;
  const int32_t* cand_count;
  const float* spec_xy;
  const uint8_t* spec_status;
  // outputs
  float* xy_out;
  int32_t* ids_out;
  int32_t* count_out;
  uint8_t* status_out;
  float* new_xy;
  int32_t* new_count;
  int32_t* next_id;
  uint8_t* occupancy;
  int32_t* stats;
};

constexpr int kRunMax = 16;   // slots (or cells) one thread owns in one pass

// One CTA per stream. Each thread owns a contiguous run of list slots (then
// of cells), so each phase is one block-wide scan of packed counts.
__global__ void __launch_bounds__(K3_THREADS) frame_finalize_kernel(K3Args a) {
  extern __shared__ int occ_s[];
  __shared__ int ws32[K3_THREADS / 32];
  __shared__ unsigned long long ws64[K3_THREADS / 32];
  const int s = blockIdx.x;
  const int n_cells = a.gx * a.gy;
  const long long cap = a.cap;
  const int t = threadIdx.x;
  for (int i = t; i < n_cells; i += K3_THREADS) occ_s[i] = 0;

  // 1. survivors of temporal tracking of both cameras, in order: counts of
  //    the two cameras packed in one int (each < 2^16)
  const int n0 = a.have_prev ? min(a.count_in[2 * s], a.cap) : 0;
  const int n1 = a.have_prev ? min(a.count_in[2 * s + 1], a.cap) : 0;
  const int run = (max(n0, n1) + K3_THREADS - 1) / K3_THREADS;
  int surv0 = 0, surv1 = 0;
  for (int r0 = 0; r0 < run; r0 += kRunMax) {
    const int rl = min(kRunMax, run - r0);
    const int first = t * run + r0;
    unsigned keep0 = 0, keep1 = 0;
    for (int j = 0; j < rl; ++j) {
      const int i = first + j;
      if (i < n0 && a.trk_status[(2LL * s) * cap + i] == VIO_TRACK_OK) keep0 |= 1u << j;
      if (i < n1 && a.trk_status[(2LL * s + 1) * cap + i] == VIO_TRACK_OK) keep1 |= 1u << j;
    }
    int tot;
    const int ex = block_scan<int>(__popc(keep0) | (__popc(keep1) << 16), ws32, tot);
    int o0 = surv0 + (ex & 0xffff), o1 = surv1 + (ex >> 16);
    for (int j = 0; j < rl; ++j) {
      const long long i0 = (2LL * s) * cap + first + j;
      if (keep0 & (1u << j)) {
        const float x = a.trk_xy[2 * i0], y = a.trk_xy[2 * i0 + 1];
        const long long d = (2LL * s) * cap + o0++;
        a.xy_out[2 * d] = x;
        a.xy_out[2 * d + 1] = y;
        a.ids_out[d] = a.ids_in[i0];
        if (x >= 0.f && y >= 0.f) {
          const int cx = cell_of(x, a.cw), cy = cell_of(y, a.ch);
          if (cx < a.gx && cy < a.gy) atomicAdd(&occ_s[cy * a.gx + cx], 1);
        }
      }
      const long long i1 = i0 + cap;
      if (keep1 & (1u << j)) {
        const long long d = (2LL * s + 1) * cap + o1++;
        a.xy_out[2 * d] = a.trk_xy[2 * i1];
        a.xy_out[2 * d + 1] = a.trk_xy[2 * i1 + 1];
        a.ids_out[d] = a.ids_in[i1];
      }
    }
    surv0 += tot & 0xffff;
    surv1 += tot >> 16;
    __syncthreads();   // ws32 is reused by the next chunk
  }
  __syncthreads();   // occupancy complete

  // 2. per cell: selection (k_eff = k - occupancy), matched subset, and the
  //    candidates matched; three counts packed in 21-bit fields
  const int id0 = a.next_id[s];
  const long long b0 = (2LL * s) * cap, b1 = b0 + cap, bn = (long long)s * cap;
  const long long cbase = (long long)s * n_cells;
  const int crun = (n_cells + K3_THREADS - 1) / K3_THREADS;
  int new_tot = 0, m_tot = 0, c_tot = 0;
  for (int r0 = 0; r0 < crun; r0 += kRunMax) {
    const int rl = min(kRunMax, crun - r0);
    const int first = t * crun + r0;
    unsigned long long packed = 0;
    for (int j = 0; j < rl; ++j) {
      const int cell = first + j;
      if (cell >= n_cells) break;
      const int nc = a.cand_count[cbase + cell];
      const int occ = min(occ_s[cell], 255);
      a.occupancy[cbase + cell] = (uint8_t)occ;
      const int nsel = max(0, min(a.k - occ, nc));
      int nm = 0;
      for (int r = 0; r < nsel; ++r)
        nm += a.spec_status[(cbase + cell) * a.k + r] == VIO_TRACK_OK;
      packed += (unsigned long long)nsel | ((unsigned long long)nm << 21) |
                ((unsigned long long)nc << 42);
    }
    unsigned long long tot;
    const unsigned long long ex = block_scan<unsigned long long>(packed, ws64, tot);
    int o = new_tot + (int)(ex & 0x1fffff);
    int om = m_tot + (int)((ex >> 21) & 0x1fffff);
    for (int j = 0; j < rl; ++j) {
      const int cell = first + j;
      if (cell >= n_cells) break;
      const int occ = min(occ_s[cell], 255);
      const int nsel = max(0, min(a.k - occ, (int)a.cand_count[cbase + cell]));
      for (int r = 0; r < nsel; ++r, ++o) {
        const long long q = (cbase + cell) * a.k + r;
        const unsigned idx = ~(unsigned)(a.cand[q] & 0xffffffffu);
        const float x = (float)(idx % (unsigned)a.W), y = (float)(idx / (unsigned)a.W);
        if (o < a.cap) {
          a.new_xy[2 * (bn + o)] = x;
          a.new_xy[2 * (bn + o) + 1] = y;
        }
        const int o0 = surv0 + o;
        if (o0 < a.cap) {
          a.xy_out[2 * (b0 + o0)] = x;
          a.xy_out[2 * (b0 + o0) + 1] = y;
          a.ids_out[b0 + o0] = id0 + o;
        }
        if (a.spec_status[q] == VIO_TRACK_OK) {
          const int o1 = surv1 + om++;
          if (o1 < a.cap) {
            a.xy_out[2 * (b1 + o1)] = a.spec_xy[2 * q];
            a.xy_out[2 * (b1 + o1) + 1] = a.spec_xy[2 * q + 1];
            a.ids_out[b1 + o1] = id0 + o;
          }
        }
      }
    }
    new_tot += (int)(tot & 0x1fffff);
    m_tot += (int)((tot >> 21) & 0x1fffff);
    c_tot += (int)((tot >> 42) & 0x1fffff);
    __syncthreads();
  }
  const int c0 = min(surv0 + new_tot, a.cap);
  const int c1 = min(surv1 + m_tot, a.cap);
  for (int i = t; i < a.cap; i += K3_THREADS) {
    a.status_out[b0 + i] = i < c0 ? VIO_TRACK_OK : VIO_TRACK_EMPTY;
    a.status_out[b1 + i] = i < c1 ? VIO_TRACK_OK : VIO_TRACK_EMPTY;
  }
  if (t == 0) {
    a.count_out[2 * s] = c0;
    a.count_out[2 * s + 1] = c1;
    a.new_count[s] = min(new_tot, a.cap);
    a.next_id[s] = id0 + new_tot;
    int32_t* st = a.stats + s * VIO_N_STATS;
    st[VIO_STAT_TRK0] = n0;
    st[VIO_STAT_TRK1] = n1;
    st[VIO_STAT_OK0] = surv0;
    st[VIO_STAT_OK1] = surv1;
    st[VIO_STAT_NEW] = new_tot;
    st[VIO_STAT_MATCHED] = m_tot;
    st[VIO_STAT_CAND] = c_tot;
  }
}

}  // namespace

cudaError_t launch_front(const vio_params& p, const Geom& g, const Batch& all, int det_step,
                         const uint8_t* mask, long long mask_stride, unsigned long long* cand,
                         int32_t* cand_count, cudaStream_t s) {
  const int gx = g.w[0] / p.cell_w, gy = g.h[0] / p.cell_h;
  K1Args a1{};
  a1.g = g;
  a1.all = all;
  a1.m = g.n_levels > 1 ? pyr::pass_levels(g.n_levels, 0) : 0;
  a1.ntx = a1.nty = 1;
  if (a1.m > 0) pyr::pass_tiles(g.w, g.h, 0, a1.m, a1.ntx, a1.nty);
  a1.det_step = det_step;
  a1.n_cells = gx * gy;
  a1.blocks_per_unit = (a1.m > 0 ? det_step * a1.ntx * a1.nty : 0) + a1.n_cells;
  a1.cg = det::CellGeom{p.cell_w, p.cell_h, gx, p.k_per_cell, p.thresholds[p.n_thresholds - 1],
                        p.detect_border};
  a1.mask = mask;
  a1.mask_stride = mask_stride;
  a1.cand = cand;
  a1.cand_count = cand_count;
  a1.round_mode = p.round_mode;
  const int smem = frame_front_smem(g, p);
  if (smem > 48 * 1024) {
    const cudaError_t e = cudaFuncSetAttribute(
        frame_front_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
  }
  const long long units = (all.n + det_step - 1) / det_step;
  const long long blocks = units * a1.blocks_per_unit;
  if (blocks > 0) frame_front_kernel<<<(unsigned)blocks, K1_THREADS, smem, s>>>(a1);
  return cudaGetLastError();
}

int frame_front_smem(const Geom& g, const vio_params& p) {
  int smem = det::cell_smem_bytes(p.cell_w, p.cell_h);
  if (g.n_levels > 1) {
    const int m = pyr::pass_levels(g.n_levels, 0);
    const int ps = pyr::pass_smem_max(g.w, g.h, 0, m);
    smem = ps > smem ? ps : smem;
  }
  return smem;
}

cudaError_t launch_frame(const FrameLaunch& f, cudaStream_t s, cudaEvent_t* marks) {
  const Geom& g = f.g;
  const int ns = f.n_streams;
  const int gx = g.w[0] / f.p.cell_w, gy = g.h[0] / f.p.cell_h;
  const int n_cells = gx * gy;
  const int k = f.p.k_per_cell;
  auto mark = [&](int i) {
    if (marks) cudaEventRecord(marks[i], s);
  };

  // K1: pyramid levels 1-4 + detection candidates (camera 0 of each stream)
  mark(0);
  cudaError_t e = launch_front(f.p, g, f.cur, 2, nullptr, 0, f.cand, f.cand_count, s);
  if (e != cudaSuccess) return e;
  // deeper pyramid levels
  mark(1);
  if (g.n_levels > 1 + pyr::kMaxPass) {
    e = launch_pyramid_from(g, f.cur, pyr::kMaxPass, f.p.round_mode, s);
    if (e != cudaSuccess) return e;
  }

  // K2: temporal tracking + stereo matching of all candidates
  mark(2);
  K2Args a2{};
  a2.g = g;
  a2.prev = f.prev;
  a2.cur = f.cur;
  a2.list_xy = f.list_xy_in;
  a2.list_count = f.list_count_in;
  a2.cap = f.cap;
  a2.n_temporal = f.have_prev ? 2LL * ns * f.cap : 0;
  a2.trk_xy = f.trk_xy;
  a2.trk_status = f.trk_status;
  a2.cand = f.cand;
  a2.cand_count = f.cand_count;
  a2.n_cells = n_cells;
  a2.k = k;
  a2.W = g.w[0];
  a2.n_stereo = (long long)ns * n_cells * k;
  a2.spec_xy = f.spec_xy;
  a2.spec_status = f.spec_status;
  a2.cfg = TrackCfg{f.p.gn_iters, 1, f.p.fb_max_dist};
  const long long warps = a2.n_temporal + a2.n_stereo;
  if (warps > 0) {
    const long long blocks2 = (warps * 32 + K2_THREADS - 1) / K2_THREADS;
    frame_track_kernel<<<(unsigned)blocks2, K2_THREADS, 0, s>>>(a2);
  }

  // K3: finalize
  mark(3);
  K3Args a3{};
  a3.have_prev = f.have_prev;
  a3.cap = f.cap;
  a3.k = k;
  a3.W = g.w[0];
  a3.gx = gx;
  a3.gy = gy;
  a3.cw = f.p.cell_w;
  a3.ch = f.p.cell_h;
  a3.trk_xy = f.trk_xy;
  a3.trk_status = f.trk_status;
  a3.ids_in = f.list_id_in;
  a3.count_in = f.list_count_in;
  a3.cand = f.cand;
  a3.cand_count = f.cand_count;
  a3.spec_xy = f.spec_xy;
  a3.spec_status = f.spec_status;
  a3.xy_out = f.list_xy_out;
  a3.ids_out = f.list_id_out;
  a3.count_out = f.list_count_out;
  a3.status_out = f.list_status;
  a3.new_xy = f.new_xy;
  a3.new_count = f.new_count;
  a3.next_id = f.next_id;
  a3.occupancy = f.occupancy;
  a3.stats = f.stats;
  const int smem3 = n_cells * (int)sizeof(int);
  if (smem3 > 48 * 1024) {
    e = cudaFuncSetAttribute(frame_finalize_kernel,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, smem3);
    if (e != cudaSuccess) return e;
  }
  frame_finalize_kernel<<<ns, K3_THREADS, smem3, s>>>(a3);
  mark(4);
  return cudaGetLastError();
}

int frame_launches(const Geom& g) {
  int n = 1;                                   // K1
  for (int s0 = pyr::kMaxPass; s0 + 1 < g.n_levels; s0 += pyr::kMaxPass) ++n;
  return n + 2;                                // K2, K3
}

}  // namespace vio
