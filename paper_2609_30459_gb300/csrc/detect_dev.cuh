// Device code of grid-cell FAST-9 detection (Sec. III-D).
//
// FAST score: with v_k the 16 ring intensities and c the centre, a bright
// 9-arc exists at tau iff the minimum of some 9 consecutive v_k exceeds
// c + tau, so the largest such tau is max_k min(v_k..v_{k+8}) - c - 1; the
// dark case is c - min_k max(v_k..v_{k+8}) - 1. Arc minima and maxima come
// from a doubling tree (pairs, quads, octets, then one more element).
//
// One CTA per (cell, image): stage the cell plus a 4-pixel halo (3 for the
// ring, 1 for the NMS neighbours), score the cell plus a 1-pixel ring, keep
// strict 3x3 maxima, and pick the cell's k strongest by k rounds of a
// block-wide maximum over packed keys (score << 32 | ~(y*w + x)): the largest
// key is the highest score, then the smallest y, then the smallest x; keys are
// unique, so each round takes the largest key below the previous winner and
// the result is deterministic. This replaces the paper's bitonic k-sort; for
// k = 1 it is its atomic-maximum variant done as a reduction.
//
// The threshold sequence collapses: the sets {score >= T} are nested and NMS
// does not depend on T, so the first T that yields k_eff keypoints gives the
// top k_eff of all maxima with score >= T_min. Pixels that cannot reach
// T_min (the paper's early rejection on the ring pairs (0,8) and (4,12): a
// 9-arc holds one point of each pair) or score below it are treated as
// non-corners: they can never win and can never suppress a pixel that scores
// >= T_min.
#pragma once
#include "common.cuh"
#include "pyramid_dev.cuh"

namespace vio {
namespace det {

constexpr int kHalo = 4;
constexpr int kThreads = 256;

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
  int best_lo = 0, best_hi = 255;
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    const int o_lo = min(q_lo[k], q_lo[(k + 4) & 15]);
    const int o_hi = max(q_hi[k], q_hi[(k + 4) & 15]);
    best_lo = max(best_lo, min(o_lo, v[(k + 8) & 15]));
    best_hi = min(best_hi, max(o_hi, v[(k + 8) & 15]));
  }
  const int m = max(best_lo - c, c - best_hi);
  return m > 0 ? m : 0;
}

// ring offsets, clockwise from the top (x right, y down)
__device__ __forceinline__ int ring_dx(int k) {
  constexpr int8_t d[16] = {0, 1, 2, 3, 3, 3, 2, 1, 0, -1, -2, -3, -3, -3, -2, -1};
  return d[k];
}
__device__ __forceinline__ int ring_dy(int k) {
  constexpr int8_t d[16] = {-3, -3, -2, -1, 0, 1, 2, 3, 3, 3, 2, 1, 0, -1, -2, -3};
  return d[k];
}

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
  v = lane < (kThreads / 32) ? red[lane] : 0ull;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long t = __shfl_xor_sync(0xffffffffu, v, o);
    v = t > v ? t : v;
  }
  return v;
}

struct CellGeom {
  int cw, ch, gx, k, tmin, border;
};

__host__ __device__ inline int cell_smem_bytes(int cw, int ch) {
  const int rs = pyr::up16(cw + 2 * kHalo + 16);
  return rs * (ch + 2 * kHalo) + (cw + 2) * (ch + 2);
}

// Detection in one cell of one image (blockDim.x == kThreads). Writes up to k
// packed keys (best first) and the count.
__device__ __forceinline__ void detect_cell(const uint8_t* __restrict__ src, int W, int H, int P,
                                            const CellGeom& cg, int cell,
                                            const uint8_t* __restrict__ mask,
                                            unsigned long long* __restrict__ out_keys,
                                            int32_t* __restrict__ out_count, uint8_t* smem,
                                            unsigned long long* red) {
  const int cy = cell / cg.gx, cx = cell - cy * cg.gx;
  const int x0 = cx * cg.cw, y0 = cy * cg.ch;
  const int rx0 = x0 - kHalo, ry0 = y0 - kHalo;
  const int xa = rx0 & ~15;
  const int RS = pyr::up16(cg.cw + 2 * kHalo + 16);
  const int MW = cg.cw + 2, MH = cg.ch + 2;
  uint8_t* reg = smem;
  uint8_t* msc = smem + RS * (cg.ch + 2 * kHalo);
  pyr::stage_rect(src, W, H, P, rx0, x0 + cg.cw + kHalo, ry0, y0 + cg.ch + kHalo, reg, RS);
  __syncthreads();

  const int T = cg.tmin;
  const Split sm(MW);
  for (int i = threadIdx.x; i < MW * MH; i += kThreads) {
    int r, c;
    sm(i, r, c);
    const int x = x0 - 1 + c, y = y0 - 1 + r;
    int m = 0;
    if (x >= 3 && x <= W - 4 && y >= 3 && y <= H - 4) {
      const uint8_t* q = reg + (y - ry0) * RS + (x - xa);
      const int ctr = q[0];
      int v[16];
#pragma unroll
      for (int k = 0; k < 16; ++k) v[k] = q[ring_dy(k) * RS + ring_dx(k)];
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

  const int b = cg.border;
  unsigned long long last = ~0ull;
  int n = 0;
  const Split sc(cg.cw);
  for (int round = 0; round < cg.k; ++round) {
    unsigned long long best = 0;
    for (int i = threadIdx.x; i < cg.cw * cg.ch; i += kThreads) {
      int r, c;
      sc(i, r, c);
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
    if (threadIdx.x == 0) out_keys[round] = best;
    last = best;
    ++n;
  }
  if (threadIdx.x == 0) *out_count = n;
}

}  // namespace det
}  // namespace vio
