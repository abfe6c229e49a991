// Grid-cell FAST-9 detection (Sec. III-D).
//
// FAST score: with v_k the 16 ring intensities and c the centre, a bright
// 9-arc exists at tau iff the minimum of some 9 consecutive v_k exceeds
// c + tau, so the largest such tau is max_k min(v_k..v_{k+8}) - c - 1; the
// dark case is c - min_k max(v_k..v_{k+8}) - 1. The arc minima and maxima
// come from a doubling tree (pairs, quads, octets, then one more element).
//
// Detection: one CTA per (cell, image). The CTA stages the cell plus a
// 4-pixel halo (3 for the ring, 1 for the NMS neighbours) in shared memory,
// scores the cell plus a 1-pixel ring, keeps strict 3x3 maxima, and picks the
// cell's k strongest by k rounds of a block-wide maximum over packed keys
// (score << 32 | ~(y*w + x)): the largest key is the highest score, then the
// smallest y, then the smallest x; keys are unique, so each round takes the
// largest key below the previous winner and the result is deterministic. This
// replaces the paper's bitonic k-sort; for k = 1 it is its atomic-maximum
// variant done as a reduction.
//
// The threshold sequence collapses: the sets {score >= T} are nested and NMS
// does not depend on T, so the first T that yields k_eff keypoints gives the
// top k_eff of all maxima with score >= T_min. Pixels that cannot reach
// T_min (early rejection on the ring pairs (0,8) and (4,12), Sec. III-D) or
// score below it are treated as non-corners: they can never win and can never
// suppress a pixel that scores >= T_min.
//
// Selection (one CTA per image) applies k_eff = k - occupancy per cell and
// writes the survivors in cell raster order with a block-wide prefix sum.
#include "common.cuh"

namespace vio {
namespace {

// Ring of the radius-3 Bresenham circle, clockwise from the top (x right,
// y down). Positions 0/8 and 4/12 are the opposite pairs used for rejection.
__constant__ int8_t kRx[16] = {0, 1, 2, 3, 3, 3, 2, 1, 0, -1, -2, -3, -3, -3, -2, -1};
__constant__ int8_t kRy[16] = {-3, -3, -2, -1, 0, 1, 2, 3, 3, 3, 2, 1, 0, -1, -2, -3};

// score + 1 in [0, 255], 0 = no corner at tau >= 0
__device__ __forceinline__ int fast_m(const int v[16], int c) {
  int p_lo[16], p_hi[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    p_lo[k] = min(v[k], v[(k + 1) & 15]);
    p_hi[k] = max(v[k], v[(k + 1) & 15]);
  }
  int q_lo[16], q_hi[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    q_lo[k] = min(p_lo[k], p_lo[(k + 2) & 15]);
    q_hi[k] = max(p_hi[k], p_hi[(k + 2) & 15]);
  }
  int best_lo = 0, best_hi = 255;   // max over arcs of the minimum; min of the maximum
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    const int o_lo = min(q_lo[k], q_lo[(k + 4) & 15]);
    const int o_hi = max(q_hi[k], q_hi[(k + 4) & 15]);
    best_lo = max(best_lo, min(o_lo, v[(k + 8) & 15]));
    best_hi = min(best_hi, max(o_hi, v[(k + 8) & 15]));
  }
  // tau_bright + 1 = best_lo - c, tau_dark + 1 = c - best_hi
  const int m = max(best_lo - c, c - best_hi);
  return m > 0 ? m : 0;
}

__global__ void fast_scores_kernel(const uint8_t* __restrict__ img, int w, int h, int pitch,
                                   int16_t* __restrict__ out) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= w || y >= h) return;
  int s = -1;
  if (x >= 3 && x <= w - 4 && y >= 3 && y <= h - 4) {
    int v[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) v[k] = __ldg(img + (long long)(y + kRy[k]) * pitch + x + kRx[k]);
    s = fast_m(v, __ldg(img + (long long)y * pitch + x)) - 1;
  }
  out[(long long)y * w + x] = (int16_t)s;
}

constexpr int DET_THREADS = 256;
constexpr int HALO = 4;

struct DetectArgs {
  Geom g;
  Batch b;
  const uint8_t* mask;
  long long mask_stride;
  unsigned long long* cand;   // [img][cell][k]
  int32_t* cand_count;        // [img][cell]
  int gx, gy, cw, ch, k, tmin, border;
};

__device__ __forceinline__ unsigned long long block_max_u64(unsigned long long v,
                                                            unsigned long long* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long t = __shfl_xor_sync(0xffffffffu, v, o);
    v = t > v ? t : v;
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();   // red[] may still be read from the previous round
  if (lane == 0) red[warp] = v;
  __syncthreads();
  v = lane < (DET_THREADS / 32) ? red[lane] : 0ull;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long t = __shfl_xor_sync(0xffffffffu, v, o);
    v = t > v ? t : v;
  }
  return v;
}

__global__ void __launch_bounds__(DET_THREADS) detect_cells_kernel(DetectArgs a) {
  extern __shared__ uint8_t smem[];
  __shared__ unsigned long long red[DET_THREADS / 32];
  const int cell = blockIdx.x, img = blockIdx.y;
  const int cy = cell / a.gx, cx = cell - cy * a.gx;
  const int W = a.g.w[0], H = a.g.h[0], P = a.g.pitch[0];
  const uint8_t* src = level_ptr(a.g, a.b, img, 0);
  const int x0 = cx * a.cw, y0 = cy * a.ch;
  const int RW = a.cw + 2 * HALO, RH = a.ch + 2 * HALO;   // staged region
  const int MW = a.cw + 2, MH = a.ch + 2;                 // scored region
  uint8_t* reg = smem;                                    // RH x RW
  uint8_t* msc = smem + RW * RH;                          // MH x MW, score + 1

  for (int i = threadIdx.x; i < RW * RH; i += DET_THREADS) {
    const int r = i / RW, c = i - r * RW;
    const int sy = min(max(y0 - HALO + r, 0), H - 1);
    const int sx = min(max(x0 - HALO + c, 0), W - 1);
    reg[i] = src[(long long)sy * P + sx];
  }
  __syncthreads();

  const int T = a.tmin;
  for (int i = threadIdx.x; i < MW * MH; i += DET_THREADS) {
    const int r = i / MW, c = i - r * MW;
    const int x = x0 - 1 + c, y = y0 - 1 + r;
    int m = 0;
    if (x >= 3 && x <= W - 4 && y >= 3 && y <= H - 4) {
      const uint8_t* q = reg + (r + HALO - 1) * RW + (c + HALO - 1);
      const int ctr = q[0];
      int v[16];
#pragma unroll
      for (int k = 0; k < 16; ++k) v[k] = q[kRy[k] * RW + kRx[k]];
      // a 9-arc holds one of each opposite pair (0,8), (4,12)
      const int hi = ctr + T, lo = ctr - T;
      const bool bright = (v[0] > hi || v[8] > hi) && (v[4] > hi || v[12] > hi);
      const bool dark = (v[0] < lo || v[8] < lo) && (v[4] < lo || v[12] < lo);
      if (bright || dark) {
        m = fast_m(v, ctr);
        if (m - 1 < T) m = 0;
      }
    }
    msc[i] = (uint8_t)m;
  }
  __syncthreads();

  const int b = a.border;
  const uint8_t* mask = a.mask ? a.mask + (long long)img * a.mask_stride : nullptr;
  unsigned long long last = ~0ull;
  unsigned long long* out = a.cand + ((long long)img * a.gx * a.gy + cell) * a.k;
  int n = 0;
  for (int round = 0; round < a.k; ++round) {
    unsigned long long best = 0;
    for (int i = threadIdx.x; i < a.cw * a.ch; i += DET_THREADS) {
      const int r = i / a.cw, c = i - r * a.cw;
      const int x = x0 + c, y = y0 + r;
      const uint8_t* q = msc + (r + 1) * MW + (c + 1);
      const int m = q[0];
      if (m == 0) continue;
      if (x < b || x > W - 1 - b || y < b || y > H - 1 - b) continue;
      const bool peak = m > q[-MW - 1] && m > q[-MW] && m > q[-MW + 1] && m > q[-1] &&
                        m > q[1] && m > q[MW - 1] && m > q[MW] && m > q[MW + 1];
      if (!peak) continue;
      if (mask && mask[(long long)y * W + x] == 0) continue;
      const unsigned long long key =
          ((unsigned long long)(m - 1) << 32) | (unsigned)(~(unsigned)(y * W + x));
      if (key < last && key > best) best = key;
    }
    best = block_max_u64(best, red);
    if (best == 0) break;
    if (threadIdx.x == 0) out[round] = best;
    last = best;
    ++n;
  }
  if (threadIdx.x == 0) a.cand_count[(long long)img * a.gx * a.gy + cell] = n;
}

constexpr int SEL_THREADS = 512;

__global__ void __launch_bounds__(SEL_THREADS) select_kernel(
    const unsigned long long* __restrict__ cand, const int32_t* __restrict__ cand_count,
    const uint8_t* __restrict__ occ, int n_cells, int k, int W, float* __restrict__ kp,
    int16_t* __restrict__ score, int32_t* __restrict__ count, int capacity) {
  __shared__ int warp_sums[SEL_THREADS / 32];
  __shared__ int carry_s;
  const int img = blockIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned long long* ci = cand + (long long)img * n_cells * k;
  const int32_t* cc = cand_count + (long long)img * n_cells;
  const uint8_t* oc = occ ? occ + (long long)img * n_cells : nullptr;
  float* kpo = kp + (long long)img * capacity * 2;
  int16_t* so = score + (long long)img * capacity;
  if (threadIdx.x == 0) carry_s = 0;
  __syncthreads();
  for (int base = 0; base < n_cells; base += SEL_THREADS) {
    const int cell = base + threadIdx.x;
    int nsel = 0;
    if (cell < n_cells) {
      const int keff = k - (oc ? (int)oc[cell] : 0);
      nsel = max(0, min(keff, (int)cc[cell]));
    }
    // block exclusive scan of nsel
    int incl = nsel;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    if (lane == 31) warp_sums[warp] = incl;
    __syncthreads();
    if (warp == 0) {
      int ws = lane < SEL_THREADS / 32 ? warp_sums[lane] : 0;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, ws, o);
        if (lane >= o) ws += t;
      }
      if (lane < SEL_THREADS / 32) warp_sums[lane] = ws;   // inclusive per warp
    }
    __syncthreads();
    const int carry = carry_s;
    const int excl = carry + (warp ? warp_sums[warp - 1] : 0) + incl - nsel;
    for (int r = 0; r < nsel; ++r) {
      const int o = excl + r;
      if (o < capacity) {
        const unsigned long long key = ci[(long long)cell * k + r];
        const unsigned idx = ~(unsigned)(key & 0xffffffffu);
        kpo[2 * o] = (float)(idx % (unsigned)W);
        kpo[2 * o + 1] = (float)(idx / (unsigned)W);
        so[o] = (int16_t)(key >> 32);
      }
    }
    __syncthreads();
    if (threadIdx.x == SEL_THREADS - 1) carry_s = carry + warp_sums[SEL_THREADS / 32 - 1];
    __syncthreads();
  }
  if (threadIdx.x == 0) count[img] = min(carry_s, capacity);
}

}  // namespace

cudaError_t launch_fast_scores(const uint8_t* img, int w, int h, int pitch, int16_t* out,
                               cudaStream_t s) {
  dim3 blk(32, 8);
  dim3 grid((w + 31) / 32, (h + 7) / 8);
  fast_scores_kernel<<<grid, blk, 0, s>>>(img, w, h, pitch, out);
  return cudaGetLastError();
}

size_t detect_smem_bytes(int cw, int ch) {
  return (size_t)(cw + 2 * HALO) * (ch + 2 * HALO) + (size_t)(cw + 2) * (ch + 2);
}

cudaError_t launch_detect(const vio_params& p, const Geom& g, const Batch& b,
                          const uint8_t* occ, const uint8_t* mask, long long mask_stride,
                          unsigned long long* cand, int32_t* cand_count, float* kp,
                          int16_t* score, int32_t* count, int capacity, cudaStream_t s) {
  DetectArgs a;
  a.g = g;
  a.b = b;
  a.mask = mask;
  a.mask_stride = mask_stride;
  a.cand = cand;
  a.cand_count = cand_count;
  a.cw = p.cell_w;
  a.ch = p.cell_h;
  a.gx = g.w[0] / p.cell_w;
  a.gy = g.h[0] / p.cell_h;
  a.k = p.k_per_cell;
  a.tmin = p.thresholds[p.n_thresholds - 1];
  a.border = p.detect_border;
  const int n_cells = a.gx * a.gy;
  if (n_cells > 0) {
    const size_t smem = detect_smem_bytes(a.cw, a.ch);
    if (smem > 48 * 1024) {
      cudaError_t e = cudaFuncSetAttribute(detect_cells_kernel,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)smem);
      if (e != cudaSuccess) return e;
    }
    dim3 grid(n_cells, b.n);
    detect_cells_kernel<<<grid, DET_THREADS, smem, s>>>(a);
  }
  select_kernel<<<b.n, SEL_THREADS, 0, s>>>(cand, cand_count, occ, n_cells, a.k, g.w[0], kp,
                                            score, count, capacity);
  return cudaGetLastError();
}

}  // namespace vio
