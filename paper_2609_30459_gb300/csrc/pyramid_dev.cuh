// Device code of the image pyramid (Sec. III-C, Eq. 1-3) and of the shared
// staging helper.
//
// A "pass" reads level s from global memory and produces levels s+1 .. s+m
// (m <= 4) for one tile, entirely in shared memory: the tile owns a
// (32 >> (m-1))-pixel square of its deepest level (the last tile of a row or
// column also owns the remainder of every level), and the region of each
// shallower level it computes follows from the filter reach, [2a-2, 2b+1) for
// an output range [a, b), clamped to the level and widened to groups of 8
// columns. Edges are replicated (Eq. 1 at the border): the staged source
// holds clamped copies, and each computed level gets copies of its edge
// columns and rows where the next level's taps fall outside it, so the
// filter itself never clamps. Each group of 8 outputs is the separable
// filter of Eq. 2-3 on 16-bit lanes (the five-row vertical sums first, then
// the horizontal one; integer sums are exact in either order) and the
// rounding shift of Eq. 3.
#pragma once
#include <algorithm>
#include <array>
#include <mutex>
#include <utility>
#include <vector>

#include "common.cuh"

namespace vio {
namespace pyr {

constexpr int kMaxPass = 4;   // levels one pass computes
constexpr int kThreads = 128;   // CTA size of the standalone pyramid launches

// deepest-level tile side of a pass of m levels: 32, 16, 8, 4, scaled by
// 2^shift (shift in -1..1), at least 1
__host__ __device__ inline int top_tile(int m, int shift = 0) {
  const int base = 32 >> (m - 1);
  const int t = shift >= 0 ? base << shift : base >> (-shift);
  return t > 0 ? t : 1;
}

struct Range {
  int s, e;   // [s, e)
};

__host__ __device__ inline int clampi(int v, int lo, int hi) {
  return v < lo ? lo : (v > hi ? hi : v);
}

// Owned range of tile index t (n tiles of side T) at a level that is `up`
// levels below the pass's deepest level (extent n_lv at that level).
__host__ __device__ inline Range owned(int t, int n_tiles, int T, int up, int n_lv) {
  const int s = (t * T) << up;
  const int e = (t == n_tiles - 1) ? n_lv : ((t + 1) * T) << up;
  return Range{s, e};
}

__host__ __device__ inline int floor_to(int v, int a) { return v >= 0 ? v / a * a : -((-v + a - 1) / a) * a; }
__host__ __device__ inline int ceil_to(int v, int a) { return -floor_to(-v, a); }
__host__ __device__ inline int up16(int v) { return (v + 15) & ~15; }

// Plan of one pass over tile (tx, ty). Index j = 0..m: level s + j (j = 0 is
// the staged source). For j >= 1, level j is computed over rows
// [ry0, ry1) (inside the level) and column groups of 8 [gx0, gx1) (multiples
// of 8, may run up to 7 columns past the level's right edge: those outputs
// are never stored). Level j < m is kept in shared memory as a buffer whose
// column 0 is image column bx (a multiple of 16) and row 0 image row by, with
// `stride` bytes per row (a multiple of 16) and `rows` rows, at byte offset
// off. Every read of the computed groups' inputs falls inside the buffer:
// a group at x0 loads bytes [2 x0 - 16, 2 x0 + 20) of rows 2y - 2 .. 2y + 2.
// Columns and rows of a buffer that lie outside its level hold replicated
// edge values where they are read as filter taps (columns -2, -1, n, n + 1
// and the same rows), so the filter needs no clamping.
struct PassPlan {
  int gx0[kMaxPass + 1], gx1[kMaxPass + 1], ry0[kMaxPass + 1], ry1[kMaxPass + 1];
  int bx[kMaxPass + 1], by[kMaxPass + 1], stride[kMaxPass + 1], rows[kMaxPass + 1];
  int off[kMaxPass + 1];
  Range ox[kMaxPass + 1], oy[kMaxPass + 1];   // owned (stored) ranges, j >= 1
  int total;                                   // shared-memory bytes
};

__host__ __device__ inline PassPlan pass_plan(const int* wl, const int* hl, int s, int m, int T,
                                              int tx, int ty, int ntx, int nty) {
  PassPlan P{};
#pragma unroll
  for (int j = 1; j <= kMaxPass; ++j) {
    if (j > m) break;
    P.ox[j] = owned(tx, ntx, T, m - j, wl[s + j]);
    P.oy[j] = owned(ty, nty, T, m - j, hl[s + j]);
  }
  // computed ranges, deepest level first: a level computes what it owns and
  // what the level above reads, clamped to the level
  int cx0 = 0, cx1 = 0, cy0 = 0, cy1 = 0;
#pragma unroll
  for (int j = kMaxPass; j >= 1; --j) {
    if (j > m) continue;
    if (j == m) {
      cx0 = P.ox[j].s;
      cx1 = P.ox[j].e;
      cy0 = P.oy[j].s;
      cy1 = P.oy[j].e;
    } else {
      cx0 = clampi(2 * P.gx0[j + 1] - 2 < P.ox[j].s ? 2 * P.gx0[j + 1] - 2 : P.ox[j].s, 0, wl[s + j]);
      cx1 = clampi(2 * P.gx1[j + 1] + 1 > P.ox[j].e ? 2 * P.gx1[j + 1] + 1 : P.ox[j].e, 0, wl[s + j]);
      cy0 = clampi(2 * P.ry0[j + 1] - 2 < P.oy[j].s ? 2 * P.ry0[j + 1] - 2 : P.oy[j].s, 0, hl[s + j]);
      cy1 = clampi(2 * P.ry1[j + 1] + 1 > P.oy[j].e ? 2 * P.ry1[j + 1] + 1 : P.oy[j].e, 0, hl[s + j]);
    }
    P.gx0[j] = floor_to(cx0, 8);
    P.gx1[j] = ceil_to(cx1, 8);
    P.ry0[j] = cy0;
    P.ry1[j] = cy1;
  }
  // buffers of levels 0 .. m-1: what level j + 1 reads, and (j >= 1) what
  // level j computes
  int off = 0;
#pragma unroll
  for (int j = 0; j < kMaxPass; ++j) {
    if (j >= m) break;
    int x0 = 2 * P.gx0[j + 1] - 16, x1 = 2 * P.gx1[j + 1] + 4;
    int y0 = 2 * P.ry0[j + 1] - 2, y1 = 2 * P.ry1[j + 1] + 1;
    if (j >= 1) {
      x0 = P.gx0[j] < x0 ? P.gx0[j] : x0;
      x1 = P.gx1[j] > x1 ? P.gx1[j] : x1;
      y0 = P.ry0[j] < y0 ? P.ry0[j] : y0;
      y1 = P.ry1[j] > y1 ? P.ry1[j] : y1;
    }
    P.bx[j] = floor_to(x0, 16);
    P.stride[j] = ceil_to(x1, 16) - P.bx[j];
    P.by[j] = y0;
    P.rows[j] = y1 - y0;
    P.off[j] = off;
    off += up16(P.stride[j] * P.rows[j]);
  }
  P.total = off;
  return P;
}

// Stages the clamped rectangle [x0, x1) x [y0, y1) of a w x h image into
// shared memory: row r at dst + r * dstride, column j <-> x = (x0 & ~15) + j.
// Interior 16-byte chunks are single vector loads when the image base and
// pitch allow it; chunks touching the image edge load byte by byte with
// replicated (clamped) coordinates.
__device__ __forceinline__ void stage_rect(const uint8_t* __restrict__ img, int w, int h,
                                           int pitch, int x0, int x1, int y0, int y1,
                                           uint8_t* dst, int dstride) {
  const int xa = x0 & ~15;
  const int nc = (x1 - xa + 15) >> 4;
  const int rows = y1 - y0;
  const bool vec_ok = ((reinterpret_cast<uintptr_t>(img) | (uintptr_t)pitch) & 15) == 0;
  const int nt = blockDim.x;
  // each thread keeps one chunk column and steps over rows (rpi rows per
  // step over the block), four rows in flight
  const int rpi = nt / nc;
  const int c = rpi > 0 ? (int)threadIdx.x % nc : (int)threadIdx.x;
  const int r0 = rpi > 0 ? (int)threadIdx.x / nc : 0;
  const int rstep = rpi > 0 ? rpi : 1;
  for (int cc = c; cc < nc; cc += (rpi > 0 ? nc : nt)) {
    if (r0 >= rstep) break;
    const int gx = xa + 16 * cc;
    const bool fast = vec_ok && gx >= 0 && gx + 16 <= w;
    uint8_t* d0 = dst + 16 * cc;
    for (int r = r0; r < rows; r += 4 * rstep) {
      uint4 v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int rr = r + u * rstep;
        if (fast && rr < rows)
          v[u] = __ldg(reinterpret_cast<const uint4*>(
              img + (long long)clampi(y0 + rr, 0, h - 1) * pitch + gx));
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int rr = r + u * rstep;
        if (rr >= rows) continue;
        uint8_t* d = d0 + rr * dstride;
        if (fast) {
          *reinterpret_cast<uint4*>(d) = v[u];
        } else {
          const uint8_t* row = img + (long long)clampi(y0 + rr, 0, h - 1) * pitch;
#pragma unroll
          for (int b = 0; b < 16; ++b) d[b] = __ldg(row + clampi(gx + b, 0, w - 1));
        }
      }
    }
  }
}

// Eq. 2 and Eq. 3 for 8 outputs of one row: level-(j) pixels x0 .. x0 + 7
// (x0 a multiple of 8) of row y, from the level below in shared memory
// (buffer `in`, column 0 = image column ibx, row 0 = image row iby, istr
// bytes per row; ibx and istr multiples of 16; every tap inside the buffer).
// Arithmetic on two 16-bit lanes per 32-bit word: the vertical sums of Eq. 2
// at the even and at the odd columns (lanes of columns c and c + 2) over the
// five rows 2y - 2 .. 2y + 2, then the horizontal sum of Eq. 3 at columns
// 2x, 2x + 1 from lane funnels, plus the rounding constant; the outputs are
// the high bytes of the lanes. Bounds: vertical sums <= 16 * 255, outputs
// <= 256 * 255 + 128 < 2^16, so no lane carries into the next.
__device__ __forceinline__ uint2 group8(const uint8_t* __restrict__ in, int istr, int ibx,
                                        int iby, int x0, int y, unsigned add2) {
  const uint8_t* p = in + (2 * y - 2 - iby) * istr + (2 * x0 - ibx);
  // E[k + 1] = vertical sums at columns (2x0 + 4k, 2x0 + 4k + 2), k = -1..4;
  // O[k + 1] = at (2x0 + 4k + 1, 2x0 + 4k + 3), k = -1..3
  unsigned E[6], O[5];
#pragma unroll
  for (int r = 0; r < 5; ++r) {
    const uint8_t* q = p + r * istr;
    const unsigned wl = *reinterpret_cast<const unsigned*>(q - 4);
    const uint4 wm = *reinterpret_cast<const uint4*>(q);
    const unsigned wr = *reinterpret_cast<const unsigned*>(q + 16);
    const unsigned w[6] = {wl, wm.x, wm.y, wm.z, wm.w, wr};
    const unsigned wt = (r == 0 || r == 4) ? 1u : (r == 2 ? 6u : 4u);
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      const unsigned e = __byte_perm(w[k], 0u, 0x4240);
      E[k] = r == 0 ? e : E[k] + wt * e;
      if (k < 5) {
        const unsigned o = __byte_perm(w[k], 0u, 0x4341);
        O[k] = r == 0 ? o : O[k] + wt * o;
      }
    }
  }
  // output lanes (x0 + 2i, x0 + 2i + 1): V(2x-2) + 4 V(2x-1) + 6 V(2x) +
  // 4 V(2x+1) + V(2x+2)
  unsigned out[4];
  unsigned A = __byte_perm(E[0], E[1], 0x5432);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const unsigned C = __byte_perm(E[i + 1], E[i + 2], 0x5432);
    const unsigned D = __byte_perm(O[i], O[i + 1], 0x5432);
    out[i] = A + C + 6u * E[i + 1] + 4u * (D + O[i + 1]) + add2;
    A = C;
  }
  return make_uint2(__byte_perm(out[0], out[1], 0x7531), __byte_perm(out[2], out[3], 0x7531));
}

// One pyramid pass for tile (tx, ty) of image img: stages level s and writes
// levels s+1..s+m (m <= kMaxPass) to global memory. All threads of the block
// must call it; `smem` is 16-byte aligned and holds pass_plan(...).total bytes.
__device__ __forceinline__ void pyramid_pass(const Geom& g, const Batch& b, int img, int s,
                                             int m, int T, int tx, int ty, int ntx, int nty,
                                             int round_mode, uint8_t* smem) {
  __shared__ PassPlan plan;
  if (threadIdx.x == 0) plan = pass_plan(g.w, g.h, s, m, T, tx, ty, ntx, nty);
  __syncthreads();
  const PassPlan& P = plan;
  stage_rect(level_ptr(g, b, img, s), g.w[s], g.h[s], g.pitch[s], P.bx[0],
             P.bx[0] + P.stride[0], P.by[0], P.by[0] + P.rows[0], smem + P.off[0], P.stride[0]);
  __syncthreads();
  const unsigned add2 = round_mode == 0 ? 0x00800080u : 0u;
#pragma unroll
  for (int j = 1; j <= kMaxPass; ++j) {
    if (j > m) break;
    const uint8_t* in = smem + P.off[j - 1];
    const int istr = P.stride[j - 1], ibx = P.bx[j - 1], iby = P.by[j - 1];
    const int ng = (P.gx1[j] - P.gx0[j]) >> 3, nr = P.ry1[j] - P.ry0[j];
    const int nw = g.w[s + j], nh = g.h[s + j];
    uint8_t* dst = level_ptr_mut(g, b, img, s + j);
    const int dpitch = g.pitch[s + j];
    const bool vec = ((reinterpret_cast<uintptr_t>(dst) | (uintptr_t)dpitch) & 7) == 0;
    const Range ox = P.ox[j], oy = P.oy[j];
    uint8_t* ob = smem + P.off[j];
    const int ostr = P.stride[j];
    // each thread keeps one group column and steps over rows
    const int nt = blockDim.x;
    const int rpi = ng > 0 ? nt / ng : 0;
    const int gstep = rpi > 0 ? ng : nt, rstep = rpi > 0 ? rpi : 1;
    const int g0 = rpi > 0 ? (int)threadIdx.x % ng : (int)threadIdx.x;
    const int r0 = rpi > 0 ? (int)threadIdx.x / ng : 0;
    for (int gi = g0; gi < ng && r0 < rstep; gi += gstep)
    for (int r = r0; r < nr; r += rstep) {
      const int y = P.ry0[j] + r, x0 = P.gx0[j] + 8 * gi;
      const uint2 v = group8(in, istr, ibx, iby, x0, y, add2);
      if (j < m) *reinterpret_cast<uint2*>(ob + (y - P.by[j]) * ostr + (x0 - P.bx[j])) = v;
      if (y >= oy.s && y < oy.e) {
        uint8_t* d = dst + (long long)y * dpitch + x0;
        if (vec && x0 >= ox.s && x0 + 8 <= ox.e) {
          *reinterpret_cast<uint2*>(d) = v;
        } else {
#pragma unroll
          for (int c = 0; c < 8; ++c)
            if (x0 + c >= ox.s && x0 + c < ox.e)
              d[c] = (uint8_t)((c < 4 ? v.x : v.y) >> (8 * (c & 3)));
        }
      }
    }
    __syncthreads();
    if (j == m) break;
    // replicated edges of this level where the next one reads them as taps:
    // columns -2, -1 (copies of column 0) and nw, nw + 1 (of column nw - 1)
    // on the computed rows, then rows -2, -1 and nh, nh + 1 (whole buffer rows)
    const int bx = P.bx[j], by = P.by[j], brows = P.rows[j];
    const bool left = bx < 0 && P.gx0[j] == 0;
    const bool right = bx + ostr > nw && P.gx1[j] >= nw;
    if (left || right) {
      for (int i = threadIdx.x; i < 4 * nr; i += blockDim.x) {
        const int y = P.ry0[j] + (i >> 2), c = i & 3;
        uint8_t* row = ob + (y - by) * ostr - bx;        // row[x] = column x
        if (c < 2) {
          if (left && -2 + c >= bx) row[-2 + c] = row[0];
        } else {
          const int x = nw + (c - 2);
          if (right && x < bx + ostr) row[x] = row[nw - 1];
        }
      }
      __syncthreads();
    }
    const bool top = by < 0 && P.ry0[j] == 0;
    const bool bottom = by + brows > nh && P.ry1[j] == nh;
    if (top || bottom) {
      const int chunks = ostr >> 4;
      for (int i = threadIdx.x; i < 4 * chunks; i += blockDim.x) {
        const int which = i / chunks, c = i - which * chunks;
        const int y = which < 2 ? -2 + which : nh + (which - 2);
        const int from = which < 2 ? 0 : nh - 1;
        if (y < by || y >= by + brows || (which < 2 ? !top : !bottom)) continue;
        reinterpret_cast<uint4*>(ob + (y - by) * ostr)[c] =
            reinterpret_cast<const uint4*>(ob + (from - by) * ostr)[c];
      }
      __syncthreads();
    }
  }
}

// Tile counts of a pass that ends at level s + m.
__host__ __device__ inline void pass_tiles(const int* wl, const int* hl, int s, int m, int T,
                                           int& ntx, int& nty) {
  ntx = (wl[s + m] + T - 1) / T;
  nty = (hl[s + m] + T - 1) / T;
}

// Passes of the standalone pyramid launches (vio_pyramid_build and the levels
// a fused launch leaves): two levels each, deepest-level tiles of 32 pixels
// (a 128 x 128 source region per tile keeps the halo recompute small).
constexpr int kRestPass = 2;
constexpr int kRestShift = 1;
__host__ __device__ inline int rest_pass_levels(int n_levels, int s) {
  const int m = n_levels - 1 - s;
  return m < kRestPass ? m : kRestPass;
}
__host__ __device__ inline int rest_passes(int rest) { return (rest + kRestPass - 1) / kRestPass; }

// Levels of the pass that starts at level s (at most kMaxPass).
__host__ __device__ inline int pass_levels(int n_levels, int s) {
  const int m = n_levels - 1 - s;
  return m < kMaxPass ? m : kMaxPass;
}

// Largest shared memory a pass over this geometry needs, over every tile.
// A tile's columns depend only on tx and its rows only on ty, so the buffer
// strides are taken per tile column and the row counts per tile row; results
// are cached per geometry (the launchers ask at every step).
inline int pass_smem_max(const int* wl, const int* hl, int s, int m, int T) {
  int ntx, nty;
  pass_tiles(wl, hl, s, m, T, ntx, nty);
  const long long key[5] = {((long long)wl[s] << 32) | (unsigned)hl[s], s, m, T,
                            ((long long)ntx << 32) | (unsigned)nty};
  static std::mutex mu;
  static std::vector<std::pair<std::array<long long, 5>, int>> cache;
  std::lock_guard<std::mutex> lock(mu);
  for (const auto& e : cache)
    if (std::equal(e.first.begin(), e.first.end(), key)) return e.second;
  std::vector<std::array<int, kMaxPass>> st(ntx), rw(nty);
  for (int tx = 0; tx < ntx; ++tx) {
    const PassPlan P = pass_plan(wl, hl, s, m, T, tx, 0, ntx, nty);
    for (int j = 0; j < kMaxPass; ++j) st[tx][j] = j < m ? P.stride[j] : 0;
  }
  for (int ty = 0; ty < nty; ++ty) {
    const PassPlan P = pass_plan(wl, hl, s, m, T, 0, ty, ntx, nty);
    for (int j = 0; j < kMaxPass; ++j) rw[ty][j] = j < m ? P.rows[j] : 0;
  }
  int best = 0;
  for (int tx = 0; tx < ntx; ++tx)
    for (int ty = 0; ty < nty; ++ty) {
      int t = 0;
      for (int j = 0; j < m; ++j) t += up16(st[tx][j] * rw[ty][j]);
      best = t > best ? t : best;
    }
  if (cache.size() >= 64) cache.erase(cache.begin());
  std::array<long long, 5> k;
  std::copy(key, key + 5, k.begin());
  cache.emplace_back(k, best);
  return best;
}

}  // namespace pyr
}  // namespace vio
