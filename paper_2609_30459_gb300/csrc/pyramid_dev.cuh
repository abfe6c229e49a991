// Device code of the image pyramid (Sec. III-C, Eq. 1-3) and of the shared
// staging helper.
//
// A "pass" reads level s from global memory and produces levels s+1 .. s+m
// (m <= 4) for one tile, entirely in shared memory: the tile owns a
// (32 >> (m-1))-pixel square of its deepest level (the last tile of a row or
// column also owns the remainder of every level), and the region of each
// shallower level it needs follows from the filter reach, [2a-2, 2b+1) for an
// output range [a, b), clamped to the level (edges are replicated, so clamped
// indices stay inside the staged region). Each level is the separable filter
// of Eq. 2 (horizontal, into 16-bit sums) then Eq. 3 (vertical, shift by 8
// with optional rounding); tiles away from the image edges skip the clamping.
#pragma once
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

// Region of level l (extent n) needed to compute range r of level l+1,
// merged with the level's own range (if any) and clamped.
__host__ __device__ inline Range need(Range up_r, Range own, int n) {
  Range r{2 * up_r.s - 2, 2 * up_r.e + 1};
  if (own.e > own.s) {
    r.s = r.s < own.s ? r.s : own.s;
    r.e = r.e > own.e ? r.e : own.e;
  }
  r.s = clampi(r.s, 0, n);
  r.e = clampi(r.e, 0, n);
  return r;
}

// Regions of a pass over tile (tx, ty): lv[0] = source level s (staged),
// lv[1..m] computed levels.
struct PassRegions {
  Range x[kMaxPass + 1], y[kMaxPass + 1];
};

__host__ __device__ inline PassRegions pass_regions(const int* wl, const int* hl, int s, int m,
                                                    int T, int tx, int ty, int ntx, int nty) {
  PassRegions R;
  // deepest level of the pass: s + m
  R.x[m] = owned(tx, ntx, T, 0, wl[s + m]);
  R.y[m] = owned(ty, nty, T, 0, hl[s + m]);
  for (int k = m - 1; k >= 0; --k) {
    const Range ox = k > 0 ? owned(tx, ntx, T, m - k, wl[s + k]) : Range{0, 0};
    const Range oy = k > 0 ? owned(ty, nty, T, m - k, hl[s + k]) : Range{0, 0};
    R.x[k] = need(R.x[k + 1], ox, wl[s + k]);
    R.y[k] = need(R.y[k + 1], oy, hl[s + k]);
  }
  return R;
}

// Shared-memory layout of a pass: staged source (16-byte aligned rows),
// computed levels, one 16-bit horizontal-pass buffer.
struct PassSmem {
  int src_stride, src_rows;       // staged source: rows x stride bytes
  int lv_stride[kMaxPass + 1], lv_off[kMaxPass + 1];  // computed level k at lv_off[k]
  int h_off, h_elems;             // uint16 buffer
  int total;
};

__host__ __device__ inline int up16(int v) { return (v + 15) & ~15; }

__host__ __device__ inline PassSmem pass_smem(const PassRegions& R, int m) {
  PassSmem S{};
  // staged columns start at a 16-byte boundary at or below R.x[0].s
  const int xa = R.x[0].s & ~15;
  S.src_stride = up16(R.x[0].e - xa + 16);
  S.src_rows = R.y[0].e - R.y[0].s;
  int off = S.src_stride * S.src_rows;
  int hmax = 0;
  for (int k = 1; k <= m; ++k) {
    S.lv_stride[k] = up16(R.x[k].e - R.x[k].s);
    S.lv_off[k] = off;
    off += S.lv_stride[k] * (R.y[k].e - R.y[k].s);
    const int h = (R.y[k - 1].e - R.y[k - 1].s) * (R.x[k].e - R.x[k].s);
    hmax = h > hmax ? h : hmax;
  }
  S.h_off = up16(off);
  S.h_elems = hmax;
  S.total = S.h_off + 2 * hmax;
  return S;
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
  const int total = nc * rows;
  const bool vec_ok = ((reinterpret_cast<uintptr_t>(img) | (uintptr_t)pitch) & 15) == 0;
  const Split sp(nc);
  for (int base = threadIdx.x; base < total; base += 4 * blockDim.x) {
    uint4 v[4];
    bool fast[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int i = base + u * blockDim.x;
      fast[u] = false;
      if (i < total) {
        int r, c;
        sp(i, r, c);
        const int gx = xa + 16 * c;
        const int gy = clampi(y0 + r, 0, h - 1);
        if (vec_ok && gx >= 0 && gx + 16 <= w) {
          v[u] = __ldg(reinterpret_cast<const uint4*>(img + (long long)gy * pitch + gx));
          fast[u] = true;
        }
      }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int i = base + u * blockDim.x;
      if (i >= total) continue;
      int r, c;
      sp(i, r, c);
      uint8_t* d = dst + r * dstride + 16 * c;
      if (fast[u]) {
        *reinterpret_cast<uint4*>(d) = v[u];
      } else {
        const int gx = xa + 16 * c;
        const uint8_t* row = img + (long long)clampi(y0 + r, 0, h - 1) * pitch;
#pragma unroll
        for (int b = 0; b < 16; ++b) d[b] = __ldg(row + clampi(gx + b, 0, w - 1));
      }
    }
  }
}

// One pyramid pass for tile (tx, ty) of image img: stages level s and writes
// levels s+1..s+m (m <= kMaxPass) to global memory. All threads of the block
// must call it; `smem` is 16-byte aligned and holds pass_smem(...).total bytes.
__device__ __forceinline__ void pyramid_pass(const Geom& g, const Batch& b, int img, int s,
                                             int m, int T, int tx, int ty, int ntx, int nty,
                                             int round_mode, uint8_t* smem) {
  const PassRegions R = pass_regions(g.w, g.h, s, m, T, tx, ty, ntx, nty);
  const PassSmem S = pass_smem(R, m);
  const uint8_t* src = level_ptr(g, b, img, s);
  const int xa = R.x[0].s & ~15;
  stage_rect(src, g.w[s], g.h[s], g.pitch[s], R.x[0].s, R.x[0].e, R.y[0].s, R.y[0].e, smem,
             S.src_stride);
  __syncthreads();
  uint16_t* hbuf = reinterpret_cast<uint16_t*>(smem + S.h_off);
  const int add = round_mode == 0 ? 128 : 0;
  for (int k = 1; k <= m; ++k) {
    // source of this level: the staged level s (k == 1) or computed level k-1
    const uint8_t* in = k == 1 ? smem : smem + S.lv_off[k - 1];
    const int in_stride = k == 1 ? S.src_stride : S.lv_stride[k - 1];
    const int in_x0 = k == 1 ? xa : R.x[k - 1].s;        // image x of column 0
    const Range ix = R.x[k - 1], iy = R.y[k - 1];       // valid range of the input
    const int wi = g.w[s + k - 1], hi = g.h[s + k - 1];
    const Range ox = R.x[k], oy = R.y[k];
    const int ow = ox.e - ox.s, oh = oy.e - oy.s;
    const int irows = iy.e - iy.s;
    // taps stay inside the level: no clamping needed for this tile
    const bool inner_x = 2 * ox.s - 2 >= 0 && 2 * (ox.e - 1) + 2 <= wi - 1;
    const bool inner_y = 2 * oy.s - 2 >= 0 && 2 * (oy.e - 1) + 2 <= hi - 1;
    // Eq. 2: horizontal pass over every input row, at the even columns 2x
    const Split so(ow);
    if (inner_x) {
      const int off = 2 * ox.s - 2 - in_x0;
      for (int i = threadIdx.x; i < irows * ow; i += blockDim.x) {
        int r, c;
        so(i, r, c);
        const uint8_t* p = in + r * in_stride + off + 2 * c;
        hbuf[i] = (uint16_t)(p[0] + 4 * (p[1] + p[3]) + 6 * p[2] + p[4]);
      }
    } else {
      for (int i = threadIdx.x; i < irows * ow; i += blockDim.x) {
        int r, c;
        so(i, r, c);
        const int x = ox.s + c;
        const uint8_t* row = in + r * in_stride;
        int sum = 0;
#pragma unroll
        for (int t = -2; t <= 2; ++t) {
          const int wt = (t == 0) ? 6 : ((t == -1 || t == 1) ? 4 : 1);
          const int sx = clampi(2 * x + t, 0, wi - 1);
          sum += wt * row[sx - in_x0];
        }
        hbuf[i] = (uint16_t)sum;
      }
    }
    (void)ix;
    __syncthreads();
    // Eq. 3: vertical pass at the even rows 2y, rounding shift
    uint8_t* outl = smem + S.lv_off[k];
    const int os = S.lv_stride[k];
    uint8_t* dst = level_ptr_mut(g, b, img, s + k);
    const int dpitch = g.pitch[s + k];
    const Range wx = owned(tx, ntx, T, m - k, g.w[s + k]);
    const Range wy = owned(ty, nty, T, m - k, g.h[s + k]);
    for (int i = threadIdx.x; i < oh * ow; i += blockDim.x) {
      int r, c;
      so(i, r, c);
      const int y = oy.s + r;
      unsigned sum = 0;
      if (inner_y) {
        const uint16_t* q = hbuf + (2 * y - 2 - iy.s) * ow + c;
        sum = q[0] + 4u * (q[ow] + q[3 * ow]) + 6u * q[2 * ow] + q[4 * ow];
      } else {
#pragma unroll
        for (int t = -2; t <= 2; ++t) {
          const unsigned wt = (t == 0) ? 6u : ((t == -1 || t == 1) ? 4u : 1u);
          const int sy = clampi(2 * y + t, 0, hi - 1);
          sum += wt * hbuf[(sy - iy.s) * ow + c];
        }
      }
      const uint8_t v = (uint8_t)((sum + add) >> 8);
      if (k < m) outl[r * os + c] = v;
      const int x = ox.s + c;
      if (x >= wx.s && x < wx.e && y >= wy.s && y < wy.e) dst[(long long)y * dpitch + x] = v;
    }
    __syncthreads();
  }
}

// Tile counts of a pass that ends at level s + m.
__host__ __device__ inline void pass_tiles(const int* wl, const int* hl, int s, int m, int T,
                                           int& ntx, int& nty) {
  ntx = (wl[s + m] + T - 1) / T;
  nty = (hl[s + m] + T - 1) / T;
}

// Levels of the pass that starts at level s (at most kMaxPass).
__host__ __device__ inline int pass_levels(int n_levels, int s) {
  const int m = n_levels - 1 - s;
  return m < kMaxPass ? m : kMaxPass;
}

// Largest shared memory a pass over this geometry needs (interior and edge
// tiles).
inline int pass_smem_max(const int* wl, const int* hl, int s, int m, int T) {
  int ntx, nty;
  pass_tiles(wl, hl, s, m, T, ntx, nty);
  int best = 0;
  const int txs[3] = {0, ntx > 1 ? ntx - 2 : 0, ntx - 1};
  const int tys[3] = {0, nty > 1 ? nty - 2 : 0, nty - 1};
  for (int a = 0; a < 3; ++a)
    for (int c = 0; c < 3; ++c) {
      const PassRegions R = pass_regions(wl, hl, s, m, T, txs[a], tys[c], ntx, nty);
      const int t = pass_smem(R, m).total;
      best = t > best ? t : best;
    }
  return best;
}

}  // namespace pyr
}  // namespace vio
