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
constexpr int kThreads = 128;   // CTA size of the standalone detection launches

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

template <int NT>
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
  v = lane < (NT / 32) ? red[lane] : 0ull;
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

// Shared memory of one cell: staged image, bound map, value map, queue of
// evaluated pixels (u16) and candidate keys (u64), 16-byte aligned pieces.
struct CellSmem {
  int rs;                      // staged row stride
  int stage, ubm, val, queue, keys, total;
};
__host__ __device__ inline CellSmem cell_smem(int cw, int ch) {
  CellSmem S;
  const int mw = cw + 2, mh = ch + 2, n = mw * mh;
  S.rs = pyr::up16(cw + 2 * kHalo + 16);
  S.stage = 0;
  S.ubm = pyr::up16(S.rs * (ch + 2 * kHalo));
  S.val = S.ubm + pyr::up16(n);
  S.queue = S.val + pyr::up16(n);
  S.keys = S.queue + pyr::up16(2 * n);
  // strict 3x3 maxima never touch: at most one per 2x2 block of the cell
  S.total = S.keys + 8 * (((cw + 1) / 2) * ((ch + 1) / 2));
  return S;
}
constexpr int kMaxCellSmem = 200 * 1024;
__host__ __device__ inline int cell_smem_bytes(int cw, int ch) { return cell_smem(cw, ch).total; }

template <int NT>
__device__ __forceinline__ unsigned block_max_u32(unsigned v, unsigned* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  v = lane < (NT / 32) ? red[lane] : 0u;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Detection in one cell of one image (blockDim.x == NT). Writes up to k
// packed keys (best first) and the count.
//
// Exact branch-and-bound. A 9-arc holds one pixel of each opposite pair
// (0,8) and (4,12) (the paper's early rejection), so with m = score + 1,
//   m <= ub = max(min(max(v0,v8), max(v4,v12)) - c, c - max(min(v0,v8), min(v4,v12))).
// Every pixel gets this bound (0 where it cannot reach T_min). Exact scores
// are computed only for pixels whose bound reaches a threshold t, lowered in
// steps until at least k candidates with m >= t are known (or t reaches
// T_min + 1). After pixels with ub >= t are evaluated, every pixel with
// m >= t has its 3x3 maximum test decided: a neighbour either is evaluated
// (exact comparison) or has ub < t <= m. So the candidates with m >= t are
// exactly known, and if there are k of them, no other pixel can enter the
// top k. The value map holds the exact m where evaluated and ub elsewhere, so
// the maximum test is "m > value of all 8 neighbours" in both cases.
template <int NT>
__device__ __forceinline__ void detect_cell(const uint8_t* __restrict__ src, int W, int H, int P,
                                            const CellGeom& cg, int cell,
                                            const uint8_t* __restrict__ mask,
                                            unsigned long long* __restrict__ out_keys,
                                            int32_t* __restrict__ out_count, uint8_t* smem,
                                            unsigned long long* red64) {
  __shared__ int c_count;
  __shared__ int wtot[NT / 32];
  unsigned* red = reinterpret_cast<unsigned*>(red64);
  const int cy = cell / cg.gx, cx = cell - cy * cg.gx;
  const int x0 = cx * cg.cw, y0 = cy * cg.ch;
  const int rx0 = x0 - kHalo, ry0 = y0 - kHalo;
  const int xa = rx0 & ~15;
  const CellSmem S = cell_smem(cg.cw, cg.ch);
  const int RS = S.rs;
  const int MW = cg.cw + 2, MH = cg.ch + 2, NR = MW * MH;
  uint8_t* reg = smem + S.stage;
  uint8_t* ubm = smem + S.ubm;      // bound of m (immutable)
  uint8_t* val = smem + S.val;      // exact m where evaluated, else the bound
  uint16_t* queue = reinterpret_cast<uint16_t*>(smem + S.queue);
  unsigned long long* keys = reinterpret_cast<unsigned long long*>(smem + S.keys);
  pyr::stage_rect(src, W, H, P, rx0, x0 + cg.cw + kHalo, ry0, y0 + cg.ch + kHalo, reg, RS);
  if (threadIdx.x == 0) c_count = 0;
  __syncthreads();

  const int T = cg.tmin;
  const int b = cg.border;
  const Split sm(MW);
  // pass A: bounds, and the largest bound of the cell's eligible pixels
  unsigned umax = 0;
  for (int i = threadIdx.x; i < NR; i += NT) {
    int r, c;
    sm(i, r, c);
    const int x = x0 - 1 + c, y = y0 - 1 + r;
    int u = 0;
    if (x >= 3 && x <= W - 4 && y >= 3 && y <= H - 4) {
      const uint8_t* q = reg + (y - ry0) * RS + (x - xa);
      const int ctr = q[0];
      const int v0 = q[-3 * RS], v8 = q[3 * RS], v4 = q[3], v12 = q[-3];
      const int hi = min(max(v0, v8), max(v4, v12));
      const int lo = max(min(v0, v8), min(v4, v12));
      u = max(hi - ctr, ctr - lo);          // >= m
      if (u - 1 < T) u = 0;                  // cannot reach T_min
    }
    ubm[i] = (uint8_t)u;
    val[i] = (uint8_t)u;
    const bool in_cell = r >= 1 && r <= cg.ch && c >= 1 && c <= cg.cw && x >= b &&
                         x <= W - 1 - b && y >= b && y <= H - 1 - b &&
                         (!mask || mask[(long long)y * W + x] != 0);
    if (in_cell) umax = max(umax, (unsigned)u);
  }
  umax = block_max_u32<NT>(umax, red);
  int n_found = 0;
  if (umax > 0) {
    const int tmin1 = T + 1;   // smallest m of a candidate
    int t_prev = 256;
    int t = max((int)umax - 24, tmin1);
    int q_done = 0;            // queue entries evaluated in earlier rounds
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (;;) {
      // pass B: queue the pixels whose bound falls in [t, t_prev): count per
      // warp, offsets from the warp totals, then write (no atomics)
      int wcount = 0;
      for (int base = 0; base < NR; base += NT) {
        const int i = base + threadIdx.x;
        const bool take = i < NR && ubm[i] >= t && ubm[i] < t_prev;
        wcount += __popc(__ballot_sync(0xffffffffu, take));
      }
      if (lane == 0) wtot[warp] = wcount;
      __syncthreads();
      int off = q_done, q_end = q_done;
#pragma unroll 4
      for (int w2 = 0; w2 < NT / 32; ++w2) {
        off += w2 < warp ? wtot[w2] : 0;
        q_end += wtot[w2];
      }
      for (int base = 0; base < NR; base += NT) {
        const int i = base + threadIdx.x;
        const bool take = i < NR && ubm[i] >= t && ubm[i] < t_prev;
        const unsigned ball = __ballot_sync(0xffffffffu, take);
        if (take) queue[off + __popc(ball & ((1u << lane) - 1))] = (uint16_t)i;
        off += __popc(ball);
      }
      __syncthreads();
      // exact scores of the newly queued pixels
      for (int e = q_done + threadIdx.x; e < q_end; e += NT) {
        const int i = queue[e];
        int r, c;
        sm(i, r, c);
        const int x = x0 - 1 + c, y = y0 - 1 + r;
        const uint8_t* q = reg + (y - ry0) * RS + (x - xa);
        int v[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) v[k] = q[ring_dy(k) * RS + ring_dx(k)];
        int m = fast_m(v, q[0]);
        if (m - 1 < T) m = 0;
        val[i] = (uint8_t)m;
      }
      __syncthreads();
      // pass C: candidates with m in [t, t_prev) among everything evaluated
      for (int e = threadIdx.x; e < q_end; e += NT) {
        const int i = queue[e];
        const int m = val[i];
        if (m < t || m >= t_prev) continue;
        int r, c;
        sm(i, r, c);
        if (r < 1 || r > cg.ch || c < 1 || c > cg.cw) continue;
        const int x = x0 - 1 + c, y = y0 - 1 + r;
        if (x < b || x > W - 1 - b || y < b || y > H - 1 - b) continue;
        const uint8_t* q = val + i;
        const bool peak = m > q[-MW - 1] && m > q[-MW] && m > q[-MW + 1] && m > q[-1] &&
                          m > q[1] && m > q[MW - 1] && m > q[MW] && m > q[MW + 1];
        if (!peak) continue;
        if (mask && mask[(long long)y * W + x] == 0) continue;
        const int slot = atomicAdd(&c_count, 1);
        keys[slot] = ((unsigned long long)(m - 1) << 32) | (unsigned)(~(unsigned)(y * W + x));
      }
      __syncthreads();
      const int found = c_count;
      if (found >= cg.k || t <= tmin1) break;
      q_done = q_end;
      t_prev = t;
      t = max(t - 24, tmin1);
      __syncthreads();
    }
    // top k of the candidate keys: k rounds of a block maximum
    const int nk = c_count;
    unsigned long long last = ~0ull;
    for (int round = 0; round < cg.k; ++round) {
      unsigned long long best = 0;
      for (int e = threadIdx.x; e < nk; e += NT) {
        const unsigned long long key = keys[e];
        if (key < last && key > best) best = key;
      }
      best = block_max_u64<NT>(best, red64);
      if (best == 0) break;
      if (threadIdx.x == 0) out_keys[round] = best;
      last = best;
      ++n_found;
    }
  }
  if (threadIdx.x == 0) *out_count = n_found;
}

}  // namespace det
}  // namespace vio
