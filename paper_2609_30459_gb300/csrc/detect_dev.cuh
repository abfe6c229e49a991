// Device code of grid-cell FAST-9 detection (Sec. III-D).
//
// FAST score: with v_k the 16 ring intensities and c the centre, a bright
// 9-arc exists at tau iff the minimum of some 9 consecutive v_k exceeds
// c + tau, so the largest such tau is max_k min(v_k..v_{k+8}) - c - 1; the
// dark case is c - min_k max(v_k..v_{k+8}) - 1. Arc minima and maxima come
// from a doubling tree over the ring (pairs, then quads, ...).
//
// Per cell: the cell plus a 1-pixel ring is scored (the ring only for the
// strict 3x3 maximum test), and the cell's k strongest maxima are picked by
// packed keys (score << 32 | ~(y*w + x)): the largest key is the highest
// score, then the smallest y, then the smallest x; keys are unique, so the
// result is deterministic. This replaces the paper's bitonic k-sort; for k = 1
// it is its atomic-maximum variant done as a reduction.
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

// ---------------------------------------------------------------------------
// Grid-cell detection by groups of warps.
//
// A CTA of NT threads takes a block of bcx x bcy cells, g warps per cell
// (g * bcx * bcy <= NT / 32; g = 1 when there are many cells to fill the GPU
// with, more when a launch has few cells), and stages the block's level-0
// region with its halo once, widened to 16 bits: every 32-bit shared word
// holds two horizontally adjacent pixels, so the bound, the masks and the
// threshold windows run on two pixels per instruction (16x2 min/max are
// native on this GPU, byte-wise SIMD is not); each thread takes four pixels
// (two words) at a time.
//
// Per cell the group keeps one map over the cell and its 1-pixel ring, 16 bits
// per pixel: high byte = ub - T_min, low byte = (m - T_min) where the exact
// score m is known, the bound ub elsewhere, both clamped at 0 (0 = cannot be
// a candidate). The shift by T_min keeps every comparison of the algorithm
// (thresholds, strict maxima) and leaves 0 for "no corner >= T_min".
//
// Exact branch-and-bound. A 9-arc holds one pixel of each opposite pair
// (0,8) and (4,12) (the paper's early rejection), so with m = score + 1,
//   m <= ub = max(min(max(v0,v8), max(v4,v12)) - c, c - max(min(v0,v8), min(v4,v12))).
// Exact scores are computed only for pixels whose bound reaches a threshold
// t, lowered in steps until at least k candidates with m >= t are known (or t
// reaches T_min + 1). After every pixel with ub >= t is evaluated, every
// pixel with m >= t has its 3x3 maximum test decided: a neighbour either is
// evaluated (exact comparison) or has ub < t <= m. So the candidates with
// m >= t are exactly known, and if there are k of them no other pixel can
// enter the top k; the result is the top k (by key) of all strict maxima with
// m >= T_min + 1, whatever the schedule of t and the split over warps.

struct BlockSmem {
  int rs, rows, stage_bytes;  // staged region: row stride (bytes), rows, bytes
  int ms, mh;                 // map: row stride (16-bit elements, multiple of 4), rows
  int g;                      // warps per cell
  int qcap, kcap;             // queue and key entries per warp
  int c_map, c_cols, c_red, c_merge, per_cell;   // byte offsets in a cell's piece
  int w_queue, w_keys, per_warp;                  // byte offsets in a warp's piece
  int cells_bytes, total;
};

// bcx x bcy cells per CTA, g warps each, one staged region for the block.
__host__ __device__ inline BlockSmem block_smem(int cw, int ch, int k, int bcx, int bcy, int g) {
  BlockSmem S;
  // columns [x0 - 8, x1 + 12) from a 16-byte boundary, whole 16-byte chunks:
  // at most width + 50 bytes
  S.rs = pyr::up16(bcx * cw + 52);
  if (((S.rs >> 2) & 31) == 0) S.rs += 16;   // rows of the same column on other banks
  S.rows = bcy * ch + 2 * kHalo;
  S.stage_bytes = pyr::up16(S.rs * S.rows);
  const int ms2 = (((cw + 2) / 2 + 2) + 1) & ~1;   // words per map row (even)
  S.ms = 2 * ms2;
  S.mh = ch + 2;
  S.g = g;
  S.qcap = 384;                                    // beyond it: pass C scans the map
  S.kcap = k + 32;
  S.c_map = 16;                                    // a guard before and a row after
  S.c_cols = S.c_map + pyr::up16(2 * S.ms * (S.mh + 1));
  S.c_red = S.c_cols + pyr::up16(8 * ms2);
  S.c_merge = S.c_red + pyr::up16(4 * 2 * g);
  S.per_cell = S.c_merge + pyr::up16(8 * g * k);
  S.w_queue = 0;
  S.w_keys = pyr::up16(2 * S.qcap);
  S.per_warp = S.w_keys + pyr::up16(8 * S.kcap);
  S.cells_bytes = bcx * bcy * S.per_cell;
  S.total = S.stage_bytes + S.cells_bytes + bcx * bcy * g * S.per_warp;
  return S;
}

constexpr int kMaxDetectSmem = 227 * 1024;

// Cells per CTA and warps per cell for NT threads and a wanted g (1, 2, 4, 8;
// lowered to NT / 32 at most): bcx x bcy = (NT / 32) / g cells when that fits
// in shared memory, else fewer (the other warps idle). False if even one cell
// does not fit or the 16-bit map index overflows.
__host__ __device__ inline bool pick_block(int cw, int ch, int k, int nt, int g_want, int& bcx,
                                           int& bcy, int& g) {
  const int nw = nt / 32;
  g = g_want < 1 ? 1 : (g_want > nw ? nw : g_want);
  if (block_smem(cw, ch, k, 1, 1, 1).ms * (ch + 3) > 65535) return false;
  for (; g >= 1; g >>= 1) {
    const int nc = nw / g;
    const int shapes[3][2] = {{nc >= 4 ? 4 : nc, nc >= 4 ? nc / 4 : 1}, {2, 1}, {1, 1}};
    for (int i = 0; i < 3; ++i) {
      const int sx = shapes[i][0], sy = shapes[i][1];
      if (sx * sy > nc || sx < 1 || sy < 1) continue;
      if (block_smem(cw, ch, k, sx, sy, g).total <= kMaxDetectSmem) {
        bcx = sx;
        bcy = sy;
        return true;
      }
    }
  }
  return false;
}

// A cell size the detection kernels support (both CTA sizes).
__host__ __device__ inline bool detect_fits(int cw, int ch, int k) {
  int bx, by, g;
  return pick_block(cw, ch, k, 128, 1, bx, by, g) && pick_block(cw, ch, k, 256, 1, bx, by, g);
}

__host__ __device__ inline int detect_blocks(int gx, int gy, int bcx, int bcy) {
  return ((gx + bcx - 1) / bcx) * ((gy + bcy - 1) / bcy);
}

// Warps per cell for a launch of n_cells cells on n_sms SMs: enough warps in
// flight (about 16 per SM) to fill the GPU.
inline int warps_per_cell(long long n_cells, int n_sms) {
  const long long want = 16LL * n_sms;
  int g = 1;
  while (g < 8 && n_cells * g < want) g <<= 1;
  return g;
}

// 16-bit lane j of a pair at image x = xp + j kept iff lo <= xp + j <= hi
__device__ __forceinline__ unsigned pair_mask(int xp, int lo, int hi) {
  return ((xp >= lo && xp <= hi) ? 0x0000ffffu : 0u) |
         ((xp + 1 >= lo && xp + 1 <= hi) ? 0xffff0000u : 0u);
}

// per 16-bit lane: a >= b (bit 15 of the lane), for a, b in [0, 256]
__device__ __forceinline__ unsigned ge2(unsigned a, unsigned b) {
  return (a + 0x80008000u - b) & 0x80008000u;
}

// m = score + 1 of the pixel at q (staged bytes, row stride rs), 0 if none:
// bright and dark arcs together, (v, 255 - v) in the two 16-bit lanes.
__device__ __forceinline__ int fast_m_pair(const uint8_t* q, int rs) {
  unsigned V[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    const unsigned s = q[ring_dy(k) * rs + ring_dx(k)];
    V[k] = s | ((255u - s) << 16);
  }
  unsigned P[16], Q[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) P[k] = __vminu2(V[k], V[(k + 1) & 15]);
#pragma unroll
  for (int k = 0; k < 16; ++k) Q[k] = __vminu2(P[k], P[(k + 2) & 15]);
  // arc k..k+8 = quads k, k+4 and k+5 (overlapping: min is idempotent)
  unsigned best = 0;
#pragma unroll
  for (int k = 0; k < 16; ++k)
    best = __vmaxu2(best, __vminu2(__vminu2(Q[k], Q[(k + 4) & 15]), Q[(k + 5) & 15]));
  const int c = q[0];
  const int lo = (int)(best & 0xffffu);          // max over arcs of the arc minimum
  const int hi = 255 - (int)(best >> 16);        // min over arcs of the arc maximum
  const int m = max(lo - c, c - hi);
  return m > 0 ? m : 0;
}

__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long v) {
  const unsigned hi = __reduce_max_sync(0xffffffffu, (unsigned)(v >> 32));
  const unsigned lo =
      __reduce_max_sync(0xffffffffu, (unsigned)(v >> 32) == hi ? (unsigned)v : 0u);
  return ((unsigned long long)hi << 32) | lo;
}

// The largest min(k, n) nonzero keys of keys[0, n) (distinct), best first,
// written by lane 0 to out[] (lanes agree on the count).
__device__ __forceinline__ int warp_top_keys(const unsigned long long* keys, int n, int k,
                                             unsigned long long* out) {
  const int lane = threadIdx.x & 31;
  unsigned long long last = ~0ull;
  int got = 0;
  for (int round = 0; round < k; ++round) {
    unsigned long long best = 0;
    for (int e = lane; e < n; e += 32) {
      const unsigned long long key = keys[e];
      if (key < last && key > best) best = key;
    }
    best = warp_max_u64(best);
    if (best == 0) break;
    if (lane == 0) out[round] = best;
    last = best;
    ++got;
  }
  return got;
}

struct CellGeom {
  int cw, ch, gx, k, tmin, border;
  int bcx, bcy, g;   // cells per CTA, warps per cell
};

// Synchronises the g warps of a cell (named barrier `bar` in 1..4, or the
// warp). Constant barrier ids keep the kernel's barrier count at 5, which
// bounds how many CTAs an SM can hold.
__device__ __forceinline__ void group_sync(int g, int bar) {
  if (g == 1) {
    __syncwarp();
    return;
  }
  const int n = 32 * g;
  switch (bar) {
    case 1: asm volatile("bar.sync 1, %0;" ::"r"(n) : "memory"); break;
    case 2: asm volatile("bar.sync 2, %0;" ::"r"(n) : "memory"); break;
    case 3: asm volatile("bar.sync 3, %0;" ::"r"(n) : "memory"); break;
    default: asm volatile("bar.sync 4, %0;" ::"r"(n) : "memory"); break;
  }
}

// Exact scores of queue entries [e0, e1) (one per lane) into the map's low
// bytes.
__device__ __forceinline__ void eval_entries(const uint16_t* queue, int e0, int e1,
                                             const uint8_t* st, int rs, int srow0, int c0,
                                             const Split& sm, int T, uint8_t* map8) {
  const int e = e0 + (threadIdx.x & 31);
  if (e < e1) {
    const int idx = queue[e];
    int r, c;
    sm(idx, r, c);
    const int m = fast_m_pair(st + (srow0 + r) * rs + c0 + c, rs);
    map8[2 * idx] = (uint8_t)max(m - T, 0);
  }
}

// Detection in one cell by warp gw of its g warps. st: the block's staged
// region (16-bit pixels, row stride rs, column 0 at image x sxa, row 0 at
// image y sy0). Writes up to k packed keys (best first) and the count.
template <bool MASKED>
__device__ __forceinline__ void detect_cell(const uint8_t* __restrict__ st, int rs, int sxa,
                                            int sy0, int W, int H, const CellGeom& cg, int cx,
                                            int cy, int gw, int bar,
                                            const uint8_t* __restrict__ mask,
                                            unsigned long long* __restrict__ out_keys,
                                            int32_t* __restrict__ out_count, uint8_t* csm,
                                            uint8_t* wsm, const BlockSmem& S) {
  const unsigned FULL = 0xffffffffu;
  const int G = S.g, GT = 32 * G;
  const int lane = threadIdx.x & 31, tg = gw * 32 + lane;
  const int cw = cg.cw, ch = cg.ch, T = cg.tmin, b = cg.border, k = cg.k;
  const int x0 = cx * cw, y0 = cy * ch;
  const int pa = ((x0 - 1 - sxa) >> 1) & ~1;                // staged pair of map column 0 (even)
  const int nq = (((x0 + cw - sxa) >> 1) - pa + 2) >> 1;     // quads (two pairs) per map row
  const int mx0 = sxa + 2 * pa;                              // image x of map column 0
  const int MH = ch + 2, MS = S.ms, MQ = S.ms >> 2;          // map quads per row
  const int srow0 = y0 - 1 - sy0;                            // staged row of map row 0
  const int rw = rs >> 2;                                    // staged words per row
  const unsigned* st32 = reinterpret_cast<const unsigned*>(st);
  uint2* map64 = reinterpret_cast<uint2*>(csm + S.c_map);
  uint8_t* map8 = csm + S.c_map;
  unsigned* colm = reinterpret_cast<unsigned*>(csm + S.c_cols);   // [pair]: ring, cell masks
  int* red = reinterpret_cast<int*>(csm + S.c_red);
  unsigned long long* merge = reinterpret_cast<unsigned long long*>(csm + S.c_merge);
  uint16_t* queue = reinterpret_cast<uint16_t*>(wsm + S.w_queue);
  unsigned long long* keys = reinterpret_cast<unsigned long long*>(wsm + S.w_keys);

  // per pair column: lanes where the bound is defined (FAST ring inside the
  // image, inside the cell's ring region) and lanes inside the cell
  for (int p = tg; p < 2 * nq; p += GT) {
    const int xp = mx0 + 2 * p;
    colm[2 * p] = pair_mask(xp, max(x0 - 1, 3), min(x0 + cw, W - 4));
    colm[2 * p + 1] = pair_mask(xp, max(x0, b), min(x0 + cw - 1, W - 1 - b));
  }
  group_sync(G, bar);

  // this thread's quads: i = tg + j * GT -> (row r, quad q), stepped without divisions
  const int n_items = MH * nq;
  const int dr = GT / nq, dq = GT - dr * nq;
  const int r_start = tg / nq, q_start = tg - r_start * nq;

  // pass A: bounds of the cell and its ring, the largest of the cell's
  const unsigned K = (0x100u + (unsigned)T) * 0x00010001u;
  unsigned acc = 0;
  {
    int r = r_start, q = q_start;
    for (int i = tg; i < n_items; i += GT) {
      const int y = y0 - 1 + r;
      const unsigned* sq = st32 + (srow0 + r) * rw + (pa >> 1) + q;   // pixels x .. x+3
      const unsigned Cw = sq[0], Uw = sq[-3 * rw], Dw = sq[3 * rw], Lw = sq[-1], Rw = sq[1];
      const uint2 C = make_uint2(__byte_perm(Cw, 0u, 0x4140), __byte_perm(Cw, 0u, 0x4342));
      const uint2 U = make_uint2(__byte_perm(Uw, 0u, 0x4140), __byte_perm(Uw, 0u, 0x4342));
      const uint2 D = make_uint2(__byte_perm(Dw, 0u, 0x4140), __byte_perm(Dw, 0u, 0x4342));
      const unsigned V12a = __byte_perm(Lw, 0u, 0x4241);                  // x - 3, x - 2
      const unsigned V12b = __byte_perm(Lw, Cw, 0x0403) & 0x00ff00ffu;    // x - 1, x
      const unsigned V4a = __byte_perm(Cw, Rw, 0x0403) & 0x00ff00ffu;     // x + 3, x + 4
      const unsigned V4b = __byte_perm(Rw, 0u, 0x4241);                   // x + 5, x + 6
      const unsigned hia = __vminu2(__vmaxu2(U.x, D.x), __vmaxu2(V4a, V12a));
      const unsigned loa = __vmaxu2(__vminu2(U.x, D.x), __vminu2(V4a, V12a));
      const unsigned hib = __vminu2(__vmaxu2(U.y, D.y), __vmaxu2(V4b, V12b));
      const unsigned lob = __vmaxu2(__vminu2(U.y, D.y), __vminu2(V4b, V12b));
      // 0x100 + max(hi - c, c - lo) per lane, then max(ub - T, 0)
      const unsigned da = __vmaxu2(hia + 0x01000100u - C.x, C.x + 0x01000100u - loa);
      const unsigned db = __vmaxu2(hib + 0x01000100u - C.y, C.y + 0x01000100u - lob);
      const uint4 cm = reinterpret_cast<const uint4*>(colm)[q];
      const bool yf = y >= 3 && y <= H - 4;
      const unsigned ua = (__vmaxu2(da, K) - K) & (yf ? cm.x : 0u);
      const unsigned ub = (__vmaxu2(db, K) - K) & (yf ? cm.z : 0u);
      map64[r * MQ + q] = make_uint2(ua * 0x0101u, ub * 0x0101u);
      const bool yc = (unsigned)(r - 1) < (unsigned)ch && y >= b && y <= H - 1 - b;
      unsigned ca = ua & (yc ? cm.y : 0u), cb = ub & (yc ? cm.w : 0u);
      if (MASKED && (ca | cb)) {   // only in-cell pixels are read
        const uint8_t* mr = mask + (long long)y * W + mx0 + 4 * q;
        ca &= ((ca & 0xffffu) && mr[0] ? 0x0000ffffu : 0u) | ((ca >> 16) && mr[1] ? 0xffff0000u : 0u);
        cb &= ((cb & 0xffffu) && mr[2] ? 0x0000ffffu : 0u) | ((cb >> 16) && mr[3] ? 0xffff0000u : 0u);
      }
      acc = __vmaxu2(acc, __vmaxu2(ca, cb));
      q += dq;
      r += dr;
      if (q >= nq) {
        q -= nq;
        ++r;
      }
    }
  }
  int umax = (int)__reduce_max_sync(FULL, max(acc & 0xffffu, acc >> 16));
  if (G > 1) {
    if (lane == 0) red[gw] = umax;
    group_sync(G, bar);
    umax = 0;
    for (int j = 0; j < G; ++j) umax = max(umax, red[j]);
  }
  group_sync(G, bar);

  const Split sm(MS);
  const unsigned lt_mask = (1u << lane) - 1u;
  const int c0 = 2 * pa;       // staged column of map column 0
  int nk = 0, q_end = 0, q_eval = 0, fw = 0;
  bool overflow = false;   // the queue lost evaluated pixels
  if (umax > 0) {
    int tp = 256;              // t_prev, above every shifted value
    int t = max(umax - 24, 1);
    for (;;) {
      const unsigned t2 = (unsigned)t * 0x00010001u, tp2 = (unsigned)tp * 0x00010001u;
      // pass B: queue this warp's pixels whose bound is in [t, tp); exact
      // scores 32 at a time
      {
        int r = r_start, q = q_start;
        for (int base = gw * 32; base < n_items; base += GT) {
          const int i = base + lane;
          unsigned ha = 0, hb = 0;
          int idx = 0;
          if (i < n_items) {
            const uint2 w = map64[r * MQ + q];
            const unsigned ua = (w.x >> 8) & 0x00ff00ffu, ub = (w.y >> 8) & 0x00ff00ffu;
            ha = ge2(ua, t2) & ~ge2(ua, tp2);
            hb = ge2(ub, t2) & ~ge2(ub, tp2);
            idx = r * MS + 4 * q;
          }
          q += dq;
          r += dr;
          if (q >= nq) {
            q -= nq;
            ++r;
          }
          const unsigned b0 = __ballot_sync(FULL, ha & 0x8000u);
          const unsigned b1 = __ballot_sync(FULL, ha & 0x80000000u);
          const unsigned b2 = __ballot_sync(FULL, hb & 0x8000u);
          const unsigned b3 = __ballot_sync(FULL, hb & 0x80000000u);
          const int total = __popc(b0) + __popc(b1) + __popc(b2) + __popc(b3);
          if (total == 0) continue;
          if (q_end + 128 > S.qcap) {   // full: score what is pending, drop the list
            eval_entries(queue, q_eval, q_end, st, rs, srow0, c0, sm, T, map8);
            __syncwarp();
            q_end = q_eval = 0;
            overflow = true;
          }
          int off = q_end + __popc(b0 & lt_mask) + __popc(b1 & lt_mask) +
                    __popc(b2 & lt_mask) + __popc(b3 & lt_mask);
          if (ha & 0x8000u) queue[off++] = (uint16_t)idx;
          if (ha & 0x80000000u) queue[off++] = (uint16_t)(idx + 1);
          if (hb & 0x8000u) queue[off++] = (uint16_t)(idx + 2);
          if (hb & 0x80000000u) queue[off] = (uint16_t)(idx + 3);
          q_end += total;
          __syncwarp();
          while (q_end - q_eval >= 32) {
            eval_entries(queue, q_eval, q_eval + 32, st, rs, srow0, c0, sm, T, map8);
            q_eval += 32;
          }
        }
        eval_entries(queue, q_eval, q_end, st, rs, srow0, c0, sm, T, map8);
        q_eval = q_end;
      }
      group_sync(G, bar);
      // pass C: evaluated pixels with a value in [t, tp) that lie in the cell
      // and exceed all 8 neighbours, from this warp's queue (or from its part
      // of the map when the queue did not hold every evaluated pixel)
      int found = 0;
      auto test = [&](int idx) -> unsigned long long {
        const int v = map8[2 * idx];
        if (v < t || v >= tp) return 0ull;
        int r, c;
        sm(idx, r, c);
        const int x = mx0 + c, y = y0 - 1 + r;
        if ((unsigned)(r - 1) >= (unsigned)ch || x < x0 || x >= x0 + cw || x < b ||
            x > W - 1 - b || y < b || y > H - 1 - b)
          return 0ull;
        const uint8_t* m = map8 + 2 * idx;
        if (!(v > m[-2] && v > m[2] && v > m[-2 * MS - 2] && v > m[-2 * MS] &&
              v > m[-2 * MS + 2] && v > m[2 * MS - 2] && v > m[2 * MS] && v > m[2 * MS + 2]))
          return 0ull;
        if (MASKED && mask[(long long)y * W + x] == 0) return 0ull;
        return ((unsigned long long)(v + T - 1) << 32) | (unsigned)(~(unsigned)(y * W + x));
      };
      auto consider = [&](unsigned long long key) {   // warp-collective append
        const unsigned bc = __ballot_sync(FULL, key != 0ull);
        if (bc == 0) return;
        const int total = __popc(bc);
        if (nk + total > S.kcap) {   // keep the k best so far (merge slot as scratch)
          const int n = warp_top_keys(keys, nk, k, merge + gw * k);
          __syncwarp();
          if (lane < n) keys[lane] = merge[gw * k + lane];
          nk = n;
          __syncwarp();
        }
        if (key) keys[nk + __popc(bc & lt_mask)] = key;
        nk += total;
        found += total;
        __syncwarp();
      };
      if (!overflow) {
        for (int base = 0; base < q_end; base += 32) {
          const int e = base + lane;
          consider(e < q_end ? test(queue[e]) : 0ull);
        }
      } else {
        int r = r_start, q = q_start;
        for (int base = gw * 32; base < n_items; base += GT) {
          const bool live = base + lane < n_items;
          const int idx0 = r * MS + 4 * q;
          q += dq;
          r += dr;
          if (q >= nq) {
            q -= nq;
            ++r;
          }
#pragma unroll 1
          for (int j = 0; j < 4; ++j) {
            const int idx = idx0 + j;
            consider(live && map8[2 * idx + 1] >= t ? test(idx) : 0ull);
          }
        }
      }
      // candidates of the whole cell (all g warps, all rounds so far)
      fw += found;
      int n_found = fw;
      if (G > 1) {
        if (lane == 0) red[G + gw] = fw;
        group_sync(G, bar);
        n_found = 0;
        for (int j = 0; j < G; ++j) n_found += red[G + j];
      }
      if (n_found >= k || t <= 1) break;
      tp = t;
      t = max(t - 24, 1);
    }
  }
  // top k of the cell: each warp's best k, then the best k of those
  if (G == 1) {
    const int n = warp_top_keys(keys, nk, k, out_keys);
    if (lane == 0) *out_count = n;
  } else {
    const int n = warp_top_keys(keys, nk, k, merge + gw * k);
    if (lane == 0)
      for (int j = n; j < k; ++j) merge[gw * k + j] = 0ull;
    group_sync(G, bar);
    if (gw == 0) {
      const int n2 = warp_top_keys(merge, G * k, k, out_keys);
      if (lane == 0) *out_count = n2;
    }
  }
}

// Detection CTA `blk` of an image: block blk (raster order over blocks of
// bcx x bcy cells), g warps per cell. All threads call it; smem holds
// block_smem(...).total bytes. MASKED: the per-pixel mask is read (non-null).
template <bool MASKED>
__device__ __forceinline__ void detect_block(const uint8_t* __restrict__ src, int W, int H, int P,
                                             const CellGeom& cg, int gy, int blk,
                                             const uint8_t* __restrict__ mask,
                                             unsigned long long* __restrict__ cand,
                                             int32_t* __restrict__ cand_count, uint8_t* smem) {
  const int nbx = (cg.gx + cg.bcx - 1) / cg.bcx;
  const int byi = blk / nbx, bxi = blk - byi * nbx;
  const int c0x = bxi * cg.bcx, c0y = byi * cg.bcy;
  const int ncx = min(cg.bcx, cg.gx - c0x), ncy = min(cg.bcy, gy - c0y);
  const int bx0 = c0x * cg.cw, bx1 = (c0x + ncx) * cg.cw;
  const int by0 = c0y * cg.ch, by1 = (c0y + ncy) * cg.ch;
  const BlockSmem S = block_smem(cg.cw, cg.ch, cg.k, cg.bcx, cg.bcy, cg.g);
  pyr::stage_rect(src, W, H, P, bx0 - 8, bx1 + 12, by0 - kHalo, by1 + kHalo, smem, S.rs);
  __syncthreads();
  const int warp = threadIdx.x >> 5;
  const int ci = warp / cg.g, gw = warp - ci * cg.g;
  const int wx = ci % cg.bcx, wy = ci / cg.bcx;
  if (wy >= cg.bcy || wx >= ncx || wy >= ncy) return;   // whole groups leave together
  const int cx = c0x + wx, cy = c0y + wy, cell = cy * cg.gx + cx;
  uint8_t* csm = smem + S.stage_bytes + ci * S.per_cell;
  uint8_t* wsm = smem + S.stage_bytes + S.cells_bytes + warp * S.per_warp;
  detect_cell<MASKED>(smem, S.rs, (bx0 - 8) & ~15, by0 - kHalo, W, H, cg, cx, cy, gw, 1 + ci,
                      mask, cand + (long long)cell * cg.k, cand_count + cell, csm, wsm, S);
}

// Fills the launch shape of cg (bcx, bcy, g) for NT threads and g_want warps
// per cell; returns the dynamic shared memory, or -1.
inline int detect_setup(CellGeom& cg, int nt, int g_want) {
  if (!pick_block(cg.cw, cg.ch, cg.k, nt, g_want, cg.bcx, cg.bcy, cg.g)) return -1;
  return block_smem(cg.cw, cg.ch, cg.k, cg.bcx, cg.bcy, cg.g).total;
}

}  // namespace det
}  // namespace vio
