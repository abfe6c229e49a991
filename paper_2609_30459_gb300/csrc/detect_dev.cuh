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
// t, which starts 24 below the largest bound of the cell and its ring and is
// lowered in steps of 24 until at least k candidates with m >= t are known
// (or t reaches T_min + 1). After every pixel with ub >= t is evaluated, every
// pixel with m >= t has its 3x3 maximum test decided: a neighbour either is
// evaluated (exact comparison) or has ub < t <= m. So the candidates with
// m >= t are exactly known, and if there are k of them no other pixel can
// enter the top k; the result is the top k (by key) of all strict maxima with
// m >= T_min + 1, whatever the schedule of t and the split over warps.

struct BlockSmem {
  int rs, rows, stage_bytes;  // staged region: row stride (bytes), rows, bytes
  int msb, mh;                // maps: row stride (bytes, multiple of 8), rows
  int g;                      // warps per cell
  int qcap, kcap;             // queue and key entries per warp
  int c_u, c_v, c_cols, c_red, c_merge, per_cell;  // byte offsets in a cell's piece
  int w_queue, w_keys, per_warp;                   // byte offsets in a warp's piece
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
  // a map row covers the cell and its ring from a 4-pixel boundary of the
  // staged region, widened to whole 8-pixel words: at most cw + 5 -> 8 * ceil
  S.msb = (cw + 5 + 7) & ~7;
  S.mh = ch + 2;
  S.g = g;
  S.qcap = 384;                                    // beyond it: pass C scans the map
  S.kcap = k + 32;
  S.c_u = 16;                                      // guards around both maps
  S.c_v = S.c_u + pyr::up16(S.msb * S.mh) + 16;
  S.c_cols = S.c_v + pyr::up16(S.msb * S.mh) + 16;
  S.c_red = S.c_cols + 8 * (S.msb / 4);
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
  if (block_smem(cw, ch, k, 1, 1, 1).msb * (ch + 2) > 65535) return false;
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

// 16-bit lanes of a pair at image x = xp (lane 0) and xp + 2 (lane 1): all
// ones in a lane iff lo <= its x <= hi
__device__ __forceinline__ unsigned pair_mask2(int xp, int lo, int hi) {
  return ((xp >= lo && xp <= hi) ? 0x0000ffffu : 0u) |
         ((xp + 2 >= lo && xp + 2 <= hi) ? 0xffff0000u : 0u);
}

// Bit 7 of each byte of the result: that byte of a >= that byte of the
// threshold tb (every byte the same t); tlo = tb & 0x7f7f7f7f. The low seven
// bits compare by a borrow-free subtraction ((a | 0x80) - (t & 0x7f) keeps
// bit 7 iff a & 0x7f >= t & 0x7f), bit 7 decides when the high bits differ.
__device__ __forceinline__ unsigned bytes_ge(unsigned a, unsigned tb, unsigned tlo) {
  const unsigned r = (a | 0x80808080u) - tlo;
  return ((a & ~tb) | (~(a ^ tb) & r)) & 0x80808080u;
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

// Top-k of a warp's keys by the cell's selection mode (VIO_SELECT_WARP_MAX or
// VIO_SELECT_BITONIC; both give the same keys).
__device__ __forceinline__ int select_top(int sel, const unsigned long long* keys, int n, int k,
                                          unsigned long long* out);

struct CellGeom {
  int cw, ch, gx, k, tmin, border;
  int bcx, bcy, g;   // cells per CTA, warps per cell
  int sel;           // VIO_SELECT_* (per-cell top-k)
};

// Bitonic sort of 64 keys, two per lane (element lane and lane + 32), into
// descending order across the warp (the paper's per-workgroup k-sort): for
// each merge size m and distance j the pair (i, i ^ j) is ordered, larger
// first where i & m == 0 (ascending blocks elsewhere, which the next merge
// turns around).
__device__ __forceinline__ void warp_bitonic64(unsigned long long& a, unsigned long long& b) {
  const unsigned lane = threadIdx.x & 31u;
#pragma unroll
  for (unsigned m = 2; m <= 64; m <<= 1) {
#pragma unroll
    for (unsigned j = m >> 1; j >= 1; j >>= 1) {
      if (j == 32) {              // pair (lane, lane + 32), both in this lane
        const bool desc = (lane & m) == 0;
        const unsigned long long hi = a > b ? a : b, lo = a > b ? b : a;
        a = desc ? hi : lo;
        b = desc ? lo : hi;
      } else {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          unsigned long long& v = h ? b : a;
          const unsigned i = lane + 32u * h;
          const unsigned long long o = __shfl_xor_sync(0xffffffffu, v, j);
          const bool lower = (i & j) == 0;          // this element is the pair's first
          const bool desc = (i & m) == 0;
          const bool keep_max = lower == desc;
          v = keep_max ? (v > o ? v : o) : (v < o ? v : o);
        }
      }
    }
  }
}

// The largest min(k, n) nonzero keys of keys[0, n) (distinct, n <= 64), best
// first, written by lane 0 to out[], by a bitonic sort; returns the count.
__device__ __forceinline__ int warp_top_keys_sorted(const unsigned long long* keys, int n, int k,
                                                    unsigned long long* out) {
  const int lane = threadIdx.x & 31;
  unsigned long long a = lane < n ? keys[lane] : 0ull;
  unsigned long long b = lane + 32 < n ? keys[lane + 32] : 0ull;
  warp_bitonic64(a, b);
  const unsigned nz = __ballot_sync(0xffffffffu, a != 0ull);
  int got = __popc(nz) + __popc(__ballot_sync(0xffffffffu, b != 0ull));
  got = got < k ? got : k;
  __syncwarp();
  if (lane < got) out[lane] = a;   // k <= 8 < 32: the best k sit in the first lanes
  __syncwarp();
  return got;
}

__device__ __forceinline__ int select_top(int sel, const unsigned long long* keys, int n, int k,
                                          unsigned long long* out) {
  return sel == VIO_SELECT_BITONIC ? warp_top_keys_sorted(keys, n, k, out)
                                   : warp_top_keys(keys, n, k, out);
}

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

// Exact scores of queue entries [e0, e1) (one per lane) into the value map.
__device__ __forceinline__ void eval_entries(const uint16_t* queue, int e0, int e1,
                                             const uint8_t* st, int rs, int srow0, int c0,
                                             const Split& sm, int T, uint8_t* vmap) {
  const int e = e0 + (threadIdx.x & 31);
  if (e < e1) {
    const int idx = queue[e];
    int r, c;
    sm(idx, r, c);
    const int m = fast_m_pair(st + (srow0 + r) * rs + c0 + c, rs);
    vmap[idx] = (uint8_t)max(m - T, 0);
  }
}

// Detection in one cell by warp gw of its g warps. st: the block's staged
// region (bytes, row stride rs, column 0 at image x sxa, a multiple of 16,
// row 0 at image y sy0). Writes up to k packed keys (best first) and the
// count.
//
// Two byte maps cover the cell and its 1-pixel ring from a 4-pixel boundary
// of the staged region (map column 0 at image x mx0), rows y0 - 1 .. y0 + ch:
//   U: ub - T_min (clamped at 0), the bound; a pixel's byte is cleared once it
//      is queued for its exact score, so each pixel is scored once;
//   V: the value the 3x3 maximum test compares: (m - T_min)+ once scored, the
//      bound before (a pixel that is not scored has ub < t <= m of any pixel
//      tested against it).
// Pass A computes the bound four pixels per thread: the 32-bit staged word
// x .. x + 3 splits into the 16-bit pairs (x, x + 2) and (x + 1, x + 3).
// Each round at threshold t scans U eight pixels per thread with byte-wise
// compares, queues the pixels whose bound reaches t and scores them 32 at a
// time; pass C then tests every scored pixel with a value in [t, tp) for a
// strict maximum in the cell.
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
  const int c0 = (x0 - 1 - sxa) & ~3;                    // staged column of map column 0
  const int mx0 = sxa + c0;                              // image x of map column 0
  const int MW = (x0 + cw + 1 - mx0 + 7) & ~7;           // map columns (multiple of 8)
  const int nq = MW >> 2, n8 = MW >> 3;                  // quads, 8-pixel words per row
  const int MH = ch + 2, MSB = S.msb;
  const int srow0 = y0 - 1 - sy0;                        // staged row of map row 0
  uint8_t* umap = csm + S.c_u;
  uint8_t* vmap = csm + S.c_v;
  uint2* colm = reinterpret_cast<uint2*>(csm + S.c_cols);   // per quad: ring masks
  int* red = reinterpret_cast<int*>(csm + S.c_red);
  unsigned long long* merge = reinterpret_cast<unsigned long long*>(csm + S.c_merge);
  uint16_t* queue = reinterpret_cast<uint16_t*>(wsm + S.w_queue);
  unsigned long long* keys = reinterpret_cast<unsigned long long*>(wsm + S.w_keys);

  // per quad: lanes where the bound is defined (FAST ring inside the image,
  // inside the cell's ring region)
  for (int q = tg; q < nq; q += GT) {
    const int xq = mx0 + 4 * q;
    const int rl = max(x0 - 1, 3), rh = min(x0 + cw, W - 4);
    colm[q] = make_uint2(pair_mask2(xq, rl, rh), pair_mask2(xq + 1, rl, rh));
  }
  const bool atomic_sel = cg.sel == VIO_SELECT_ATOMIC;   // k == 1: one 64-bit maximum per cell
  if (atomic_sel && tg == 0) merge[0] = 0ull;
  group_sync(G, bar);

  // pass A: bounds of the cell and its ring and the largest of them (it only
  // sets the first threshold: any start at or above the largest bound of the
  // cell's unmasked pixels gives the same result); this
  // thread's quads i = tg + j * GT -> (row r, quad q), stepped without divisions
  const unsigned K = (0x100u + (unsigned)T) * 0x00010001u;
  unsigned acc = 0;
  {
    const int n_items = MH * nq;
    const int dr = GT / nq, dq = GT - dr * nq;
    int r = tg / nq, q = tg - (tg / nq) * nq;
    for (int i = tg; i < n_items; i += GT) {
      const int y = y0 - 1 + r;
      const uint8_t* sq = st + (srow0 + r) * rs + c0 + 4 * q;           // pixels x .. x + 3
      const unsigned Cw = *reinterpret_cast<const unsigned*>(sq);
      const unsigned Uw = *reinterpret_cast<const unsigned*>(sq - 3 * rs);
      const unsigned Dw = *reinterpret_cast<const unsigned*>(sq + 3 * rs);
      const unsigned Lw = *reinterpret_cast<const unsigned*>(sq - 4);
      const unsigned Rw = *reinterpret_cast<const unsigned*>(sq + 4);
      // pair a = pixels (x, x + 2), pair b = (x + 1, x + 3); compass points
      // of the ring: up, down (rows -3, +3), left (x - 3), right (x + 3)
      const unsigned Ca = __byte_perm(Cw, 0u, 0x4240), Cb = __byte_perm(Cw, 0u, 0x4341);
      const unsigned Ua = __byte_perm(Uw, 0u, 0x4240), Ub = __byte_perm(Uw, 0u, 0x4341);
      const unsigned Da = __byte_perm(Dw, 0u, 0x4240), Db = __byte_perm(Dw, 0u, 0x4341);
      const unsigned La = __byte_perm(Lw, 0u, 0x4341);                     // x - 3, x - 1
      const unsigned Lb = __byte_perm(Lw, Cw, 0x0402) & 0x00ff00ffu;      // x - 2, x
      const unsigned Ra = __byte_perm(Cw, Rw, 0x0503) & 0x00ff00ffu;      // x + 3, x + 5
      const unsigned Rb = __byte_perm(Rw, 0u, 0x4240);                     // x + 4, x + 6
      const unsigned hia = __vminu2(__vmaxu2(Ua, Da), __vmaxu2(Ra, La));
      const unsigned loa = __vmaxu2(__vminu2(Ua, Da), __vminu2(Ra, La));
      const unsigned hib = __vminu2(__vmaxu2(Ub, Db), __vmaxu2(Rb, Lb));
      const unsigned lob = __vmaxu2(__vminu2(Ub, Db), __vminu2(Rb, Lb));
      // 0x100 + max(hi - c, c - lo) per lane, then max(ub - T, 0)
      const unsigned da = __vmaxu2(hia + 0x01000100u - Ca, Ca + 0x01000100u - loa);
      const unsigned db = __vmaxu2(hib + 0x01000100u - Cb, Cb + 0x01000100u - lob);
      const uint2 cm = colm[q];
      const bool yf = y >= 3 && y <= H - 4;
      const unsigned ua = (__vmaxu2(da, K) - K) & (yf ? cm.x : 0u);
      const unsigned ub = (__vmaxu2(db, K) - K) & (yf ? cm.y : 0u);
      const unsigned word = __byte_perm(ua, ub, 0x6240);                   // x .. x + 3
      *reinterpret_cast<unsigned*>(umap + r * MSB + 4 * q) = word;
      *reinterpret_cast<unsigned*>(vmap + r * MSB + 4 * q) = word;
      acc = __vmaxu2(acc, __vmaxu2(ua, ub));
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

  const Split sm(MSB);
  const unsigned lt_mask = (1u << lane) - 1u;
  int nk = 0, q_end = 0, q_eval = 0, fw = 0;
  bool overflow = false;   // the queue lost scored pixels
  if (umax > 0) {
    int tp = 256;              // t_prev, above every shifted value
    int t = max(umax - 24, 1);
    const int n_words = MH * n8;
    const int dr8 = GT / n8, dc8 = GT - dr8 * n8;
    for (;;) {
      // pass B: queue this warp's pixels whose bound reaches t (their U
      // bytes are cleared), exact scores 32 at a time
      {
        const unsigned tb = (unsigned)t * 0x01010101u, tlo = tb & 0x7f7f7f7fu;
        int r = tg / n8, c8 = tg - (tg / n8) * n8;
        for (int base = gw * 32; base < n_words; base += GT) {
          const int i = base + lane;
          uint2 w = make_uint2(0u, 0u);
          const int idx0 = r * MSB + 8 * c8;
          if (i < n_words) w = *reinterpret_cast<const uint2*>(umap + idx0);
          c8 += dc8;
          r += dr8;
          if (c8 >= n8) {
            c8 -= n8;
            ++r;
          }
          const unsigned hx = bytes_ge(w.x, tb, tlo), hy = bytes_ge(w.y, tb, tlo);
          const int cnt = __popc(hx) + __popc(hy);
          if (__ballot_sync(FULL, cnt != 0) == 0) continue;
          int incl = cnt;
#pragma unroll
          for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(FULL, incl, o);
            if (lane >= o) incl += v;
          }
          const int total = __shfl_sync(FULL, incl, 31);
          if (q_end + total > S.qcap) {   // full: score what is pending, drop the list
            eval_entries(queue, q_eval, q_end, st, rs, srow0, c0, sm, T, vmap);
            __syncwarp();
            q_end = q_eval = 0;
            overflow = true;
          }
          if (cnt) {
            int off = q_end + incl - cnt;
            for (unsigned h = hx; h; h &= h - 1) queue[off++] = (uint16_t)(idx0 + ((__ffs(h) - 1) >> 3));
            for (unsigned h = hy; h; h &= h - 1) queue[off++] = (uint16_t)(idx0 + 4 + ((__ffs(h) - 1) >> 3));
            w.x &= ~((hx >> 7) * 0xffu);
            w.y &= ~((hy >> 7) * 0xffu);
            *reinterpret_cast<uint2*>(umap + idx0) = w;
          }
          q_end += total;
          __syncwarp();
          while (q_end - q_eval >= 32) {
            eval_entries(queue, q_eval, q_eval + 32, st, rs, srow0, c0, sm, T, vmap);
            q_eval += 32;
          }
        }
        eval_entries(queue, q_eval, q_end, st, rs, srow0, c0, sm, T, vmap);
        q_eval = q_end;
      }
      group_sync(G, bar);
      // pass C: scored pixels with a value in [t, tp) that lie in the cell
      // and exceed all 8 neighbours, from this warp's queue (or from the map
      // words this warp scans, when its queue did not hold every pixel it
      // scored: a pixel with a value >= t has been scored)
      int found = 0;
      auto test = [&](int idx) -> unsigned long long {
        const int v = vmap[idx];
        if (v < t || v >= tp) return 0ull;
        int r, c;
        sm(idx, r, c);
        const int x = mx0 + c, y = y0 - 1 + r;
        if ((unsigned)(r - 1) >= (unsigned)ch || x < x0 || x >= x0 + cw || x < b ||
            x > W - 1 - b || y < b || y > H - 1 - b)
          return 0ull;
        const uint8_t* m = vmap + idx;
        if (!(v > m[-1] && v > m[1] && v > m[-MSB - 1] && v > m[-MSB] && v > m[-MSB + 1] &&
              v > m[MSB - 1] && v > m[MSB] && v > m[MSB + 1]))
          return 0ull;
        if (MASKED && mask[(long long)y * W + x] == 0) return 0ull;
        return ((unsigned long long)(v + T - 1) << 32) | (unsigned)(~(unsigned)(y * W + x));
      };
      auto consider = [&](unsigned long long key) {   // warp-collective append
        const unsigned bc = __ballot_sync(FULL, key != 0ull);
        if (bc == 0) return;
        const int total = __popc(bc);
        if (atomic_sel) {
          if (key) atomicMax(merge, key);
          found += total;
          return;
        }
        if (nk + total > S.kcap) {   // keep the k best so far (merge slot as scratch)
          const int n = select_top(cg.sel, keys, nk, k, merge + gw * k);
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
        // the 8-pixel words this warp scanned in pass B (the pixels it queued)
        int r = tg / n8, c8 = tg - (tg / n8) * n8;
        for (int base = gw * 32; base < n_words; base += GT) {
          const bool live = base + lane < n_words;
          const int idx0 = r * MSB + 8 * c8;
          c8 += dc8;
          r += dr8;
          if (c8 >= n8) {
            c8 -= n8;
            ++r;
          }
#pragma unroll 1
          for (int j = 0; j < 8; ++j) consider(live ? test(idx0 + j) : 0ull);
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
  // top k of the cell: each warp's best k, then the best k of those (or,
  // with the atomic maximum, the cell's one slot)
  if (atomic_sel) {
    group_sync(G, bar);
    if (tg == 0) {
      const unsigned long long best = merge[0];
      if (best) out_keys[0] = best;
      *out_count = best ? 1 : 0;
    }
  } else if (G == 1) {
    const int n = select_top(cg.sel, keys, nk, k, out_keys);
    if (lane == 0) *out_count = n;
  } else {
    const int n = select_top(cg.sel, keys, nk, k, merge + gw * k);
    if (lane == 0)
      for (int j = n; j < k; ++j) merge[gw * k + j] = 0ull;
    group_sync(G, bar);
    if (gw == 0) {
      const int n2 = select_top(cg.sel, merge, G * k, k, out_keys);
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
