// Device code of the patch tracker (Sec. III-E, Eq. 4-5): one warp of 32
// threads per keypoint, each lane owning up to two of the 52 pattern points.
//
// Algebra used on the device. With raw template samples s_i, raw gradients
// g_i and J'_i = [g_x, g_y, g_y u_i - g_x v_i], the mean-normalised
// quantities of Eq. 4 are J_i = J'_i / Ibar, H = H' / Ibar^2 (H' = sum
// J'_i^T J'_i) and G_i = Ibar H'^-1 J'_i, so Eq. 5's increment
//   delta = -sum_i G_i (r_i / rbar - s_i / Ibar)
// equals  delta = c - (S / R) k,  with S = sum s_i, R = sum r_i,
// c = H'^-1 sum J'_i s_i (per template) and k = sum (H'^-1 J'_i) r_i (per
// iteration). Each Gauss-Newton step therefore needs ONE warp reduction of
// four values (R, k), not two dependent ones.
//
// Positions keep an integer anchor plus a small float offset, so bilinear
// weights carry full FP32 precision at any image size; template samples of
// one keypoint share one sub-pixel offset and therefore one set of weights.
// The rotation is carried as (cos, sin) and updated by the increment's
// rotation, whose cosine, sine and the SE(2) left-Jacobian terms come from
// their Taylor series for small angles (|phi| < 0.25, error < 1e-9), so a
// Gauss-Newton step evaluates no trigonometric function.
//
// Every product that meets a sum is written as an explicit FMA (__fmaf_rn)
// or an unfused product (__fmul_rn), so the rounding of each expression is
// fixed in the source rather than by the compiler's contraction in each
// kernel that inlines this code: all tracking kernels and launch shapes give
// bit-identical results.
#pragma once
#include <math.h>

#include "common.cuh"

namespace vio {
namespace trk {

// The sample pattern (Sec. III-E gives only its size, 52): the odd lattice
// u, v in {+-1, +-3, +-5, +-7} with |u| + |v| <= 10, ordered by v then u.
struct Pattern {
  int8_t u[kPatternMax], v[kPatternMax];
  int n;
};
constexpr Pattern make_pattern() {
  Pattern p{};
  int n = 0;
  for (int v = -7; v <= 7; v += 2)
    for (int u = -7; u <= 7; u += 2) {
      const int au = u < 0 ? -u : u, av = v < 0 ? -v : v;
      if (au + av <= 10) {
        p.u[n] = (int8_t)u;
        p.v[n] = (int8_t)v;
        ++n;
      }
    }
  p.n = n;
  return p;
}
static_assert(make_pattern().n == 52, "pattern size");
constexpr int kNP = 52;

// Point i of the pattern, by rows: v = -7, -5, ..., 7 hold 4, 6, 8, 8, 8, 8,
// 6, 4 points, u running from -hw to hw in steps of 2 (hw = 3, 5, 7, ...).
__host__ __device__ constexpr void point_of(int i, int& u, int& v) {
  int start = 0;
  for (int r = 0; r < 8; ++r) {
    const int hw = (r == 0 || r == 7) ? 3 : (r == 1 || r == 6) ? 5 : 7;
    const int n = hw + 1;
    if (i < start + n) {
      v = -7 + 2 * r;
      u = -hw + 2 * (i - start);
      return;
    }
    start += n;
  }
  u = v = 0;
}
constexpr bool pattern_rows_match() {
  const Pattern P = make_pattern();
  for (int i = 0; i < kNP; ++i) {
    int u = 0, v = 0;
    point_of(i, u, v);
    if (u != P.u[i] || v != P.v[i]) return false;
  }
  return true;
}
static_assert(pattern_rows_match(), "row form of the pattern");

// The lane's two pattern points (the second exists for lanes 0..19; lanes
// 20..31 evaluate the pattern's centre there, with weight w1 = 0).
struct LanePts {
  int iu[2], iv[2];
  float u[2], v[2];
  float w1;
};
__device__ __forceinline__ LanePts lane_points(int lane) {
  LanePts P;
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    const int i = lane + 32 * j;
    int u = 0, v = 0;
    if (i < kNP) point_of(i, u, v);
    P.iu[j] = u;
    P.iv[j] = v;
    P.u[j] = (float)u;
    P.v[j] = (float)v;
  }
  P.w1 = lane + 32 < kNP ? 1.f : 0.f;
  return P;
}

struct Lv {
  const uint8_t* p;
  int w, h, pitch;
};

template <int N>
__device__ __forceinline__ void warp_sum(float (&v)[N]) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
#pragma unroll
    for (int i = 0; i < N; ++i) v[i] += __shfl_xor_sync(0xffffffffu, v[i], o);
}

// Sums four values over the warp and gives every lane all four totals.
// BUTTERFLY: an xor butterfly, five rounds of four independent exchanges
// (the two lanes of every exchange add the same two operands, so partners
// hold bitwise equal partial sums after each round and every lane ends with
// the same totals): the shortest dependent chain, for launches that leave the
// GPU mostly idle. Else a transposed butterfly with half the exchanges (after
// the xor-16 and xor-8 rounds each lane carries one of the four partial sums,
// value 2*bit4 + bit3 of its lane id, three more xor rounds finish it, four
// broadcasts hand it out): fewer instructions, for launches that fill it.
template <bool BUTTERFLY>
__device__ __forceinline__ void warp_sum4(float& a0, float& a1, float& a2, float& a3) {
  if (BUTTERFLY) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float b0 = __shfl_xor_sync(0xffffffffu, a0, o);
      const float b1 = __shfl_xor_sync(0xffffffffu, a1, o);
      const float b2 = __shfl_xor_sync(0xffffffffu, a2, o);
      const float b3 = __shfl_xor_sync(0xffffffffu, a3, o);
      a0 += b0;
      a1 += b1;
      a2 += b2;
      a3 += b3;
    }
    return;
  }
  const unsigned lane = threadIdx.x & 31u;
  const bool h16 = lane & 16u, h8 = lane & 8u;
  float k0 = h16 ? a2 : a0, k1 = h16 ? a3 : a1;
  const float s0 = h16 ? a0 : a2, s1 = h16 ? a1 : a3;
  k0 += __shfl_xor_sync(0xffffffffu, s0, 16);
  k1 += __shfl_xor_sync(0xffffffffu, s1, 16);
  float k = h8 ? k1 : k0;
  k += __shfl_xor_sync(0xffffffffu, h8 ? k0 : k1, 8);
  k += __shfl_xor_sync(0xffffffffu, k, 4);
  k += __shfl_xor_sync(0xffffffffu, k, 2);
  k += __shfl_xor_sync(0xffffffffu, k, 1);
  a0 = __shfl_sync(0xffffffffu, k, 0);
  a1 = __shfl_sync(0xffffffffu, k, 8);
  a2 = __shfl_sync(0xffffffffu, k, 16);
  a3 = __shfl_sync(0xffffffffu, k, 24);
}

// position = anchor (int) + offset (float)
struct Pos {
  int ax, ay;
  float dx, dy;
};

__device__ __forceinline__ void rebase(Pos& t) {
  const float fx = floorf(t.dx), fy = floorf(t.dy);
  t.ax += (int)fx;
  t.dx -= fx;
  t.ay += (int)fy;
  t.dy -= fy;
}

// (a + d) / 2^l as anchor Q + offset f in [0, 1)
__device__ __forceinline__ void to_level1(int a, float d, int l, int& Q, float& f) {
  const int Ql = a >> l;
  const float frac = ((float)(a - Ql * (1 << l)) + d) * __int_as_float((127 - l) << 23);
  const float fl = floorf(frac);
  Q = Ql + (int)fl;
  f = frac - fl;
}

__device__ __forceinline__ Pos split(float x, float y) {
  Pos p;
  const float fx = floorf(x), fy = floorf(y);
  p.ax = (int)fx;
  p.ay = (int)fy;
  p.dx = x - fx;
  p.dy = y - fy;
  return p;
}

struct Tpl {
  float K[2][3];   // H'^-1 J'_i for the lane's two points
  float c0, c1, c2;  // H'^-1 sum J'_i s_i
  float S;         // sum s_i
};

// Cholesky factor of H' with reciprocal diagonal (no divisions in solves).
struct Chol {
  float i00, l10, l20, i11, l21, i22;   // i.. = 1 / l..
  __device__ __forceinline__ void solve(float b0, float b1, float b2, float& x0, float& x1,
                                        float& x2) const {
    const float y0 = __fmul_rn(b0, i00);
    const float y1 = __fmul_rn(__fmaf_rn(-l10, y0, b1), i11);
    const float y2 = __fmul_rn(__fmaf_rn(-l21, y1, __fmaf_rn(-l20, y0, b2)), i22);
    x2 = __fmul_rn(y2, i22);
    x1 = __fmul_rn(__fmaf_rn(-l21, x2, y1), i11);
    x0 = __fmul_rn(__fmaf_rn(-l20, x2, __fmaf_rn(-l10, x1, y0)), i00);
  }
};

// Sums N values over the warp with a transposed butterfly (N padded to 16):
// the xor-16, -8, -4, -2 exchanges halve the values each lane carries, the
// xor-1 exchange completes them (value j ends in lanes 2j and 2j+1), and N
// broadcasts return every total to every lane.
template <int N>
__device__ __forceinline__ void warp_sum_t(float (&v)[N]) {
  static_assert(N <= 16, "at most 16 values");
  const unsigned lane = threadIdx.x & 31u;
  float a[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) a[i] = i < N ? v[i] : 0.f;
#pragma unroll
  for (int half = 8, bit = 16; half >= 1; half >>= 1, bit >>= 1) {
    const bool up = lane & (unsigned)bit;
#pragma unroll
    for (int i = 0; i < half; ++i) {
      const float keep = up ? a[i + half] : a[i];
      const float send = up ? a[i] : a[i + half];
      a[i] = keep + __shfl_xor_sync(0xffffffffu, send, bit);
    }
  }
  a[0] += __shfl_xor_sync(0xffffffffu, a[0], 1);
  // lane L now holds value (L >> 1) read as bits 4..1 of L: value j is in lane 2j
#pragma unroll
  for (int i = 0; i < N; ++i) {
    // value index of lane L is its bits 4,3,2,1 in the order the rounds split
    // them: bit4 -> 8, bit3 -> 4, bit2 -> 2, bit1 -> 1
    v[i] = __shfl_sync(0xffffffffu, a[0], 2 * i);
  }
}

// Template of keypoint q (level-0 anchor form) at level l of the source.
// Returns a VIO_TRACK_* status, uniform across the warp.
__device__ __forceinline__ int build_template(const Lv& L, const Pos& q, int l, int lane,
                                              const LanePts& P, Tpl& T) {
  int Qx, Qy;
  float fx, fy;
  to_level1(q.ax, q.dx, l, Qx, fx);
  to_level1(q.ay, q.dy, l, Qy, fy);
  // bilinear at c and c +- 1 needs 1 <= c < w - 2: on integers 1 <= Q + u <= w - 3;
  // the pattern spans [-7, 7] in both axes, so the extreme points decide
  const bool ok = Qx - 7 >= 1 && Qx + 7 <= L.w - 3 && Qy - 7 >= 1 && Qy + 7 <= L.h - 3;
  if (!ok) return VIO_TRACK_OOB_TEMPLATE;   // same value in every lane

  const float w00 = __fmul_rn(1.f - fx, 1.f - fy), w10 = __fmul_rn(fx, 1.f - fy);
  const float w01 = __fmul_rn(1.f - fx, fy), w11 = __fmul_rn(fx, fy);
  float Jp[2][3];
  float acc[10];
#pragma unroll
  for (int i = 0; i < 10; ++i) acc[i] = 0.f;
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    const int i = lane + 32 * j;
    Jp[j][0] = Jp[j][1] = Jp[j][2] = 0.f;
    if (j == 0 || i < kNP) {
      const float u = P.u[j], v = P.v[j];
      const uint8_t* base =
          L.p + (long long)(Qy + P.iv[j] - 1) * L.pitch + (Qx + P.iu[j] - 1);
      float t[4][4];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int cc = 0; cc < 4; ++cc)
          t[r][cc] = (r == 0 || r == 3) && (cc == 0 || cc == 3)
                         ? 0.f
                         : (float)__ldg(base + (long long)r * L.pitch + cc);
      auto bl = [&](float a, float b, float c, float d) {
        return __fmaf_rn(w11, d, __fmaf_rn(w01, c, __fmaf_rn(w10, b, __fmul_rn(w00, a))));
      };
      const float s = bl(t[1][1], t[1][2], t[2][1], t[2][2]);
      const float gx = __fmul_rn(0.5f, bl(t[1][2], t[1][3], t[2][2], t[2][3]) -
                                            bl(t[1][0], t[1][1], t[2][0], t[2][1]));
      const float gy = __fmul_rn(0.5f, bl(t[2][1], t[2][2], t[3][1], t[3][2]) -
                                            bl(t[0][1], t[0][2], t[1][1], t[1][2]));
      Jp[j][0] = gx;
      Jp[j][1] = gy;
      const float jt = __fmaf_rn(-gx, v, __fmul_rn(gy, u));
      Jp[j][2] = jt;
      acc[0] += s;
      acc[1] = __fmaf_rn(gx, gx, acc[1]);
      acc[2] = __fmaf_rn(gx, gy, acc[2]);
      acc[3] = __fmaf_rn(gx, jt, acc[3]);
      acc[4] = __fmaf_rn(gy, gy, acc[4]);
      acc[5] = __fmaf_rn(gy, jt, acc[5]);
      acc[6] = __fmaf_rn(jt, jt, acc[6]);
      acc[7] = __fmaf_rn(gx, s, acc[7]);
      acc[8] = __fmaf_rn(gy, s, acc[8]);
      acc[9] = __fmaf_rn(jt, s, acc[9]);
    }
  }
  warp_sum_t(acc);
  T.S = acc[0];
  if (!(acc[0] > 0.f)) return VIO_TRACK_ZERO_MEAN;
  // Cholesky of H'; a pivot <= 1e-9 trace marks a degenerate patch
  const float eps = __fmul_rn(1e-9f, acc[1] + acc[4] + acc[6]);
  Chol C;
  if (!(acc[1] > eps)) return VIO_TRACK_DEGENERATE_H;
  C.i00 = rsqrtf(acc[1]);
  C.l10 = __fmul_rn(acc[2], C.i00);
  C.l20 = __fmul_rn(acc[3], C.i00);
  const float d1 = __fmaf_rn(-C.l10, C.l10, acc[4]);
  if (!(d1 > eps)) return VIO_TRACK_DEGENERATE_H;
  C.i11 = rsqrtf(d1);
  C.l21 = __fmul_rn(__fmaf_rn(-C.l20, C.l10, acc[5]), C.i11);
  const float d2 = __fmaf_rn(-C.l21, C.l21, __fmaf_rn(-C.l20, C.l20, acc[6]));
  if (!(d2 > eps)) return VIO_TRACK_DEGENERATE_H;
  C.i22 = rsqrtf(d2);
  C.solve(acc[7], acc[8], acc[9], T.c0, T.c1, T.c2);
#pragma unroll
  for (int j = 0; j < 2; ++j) C.solve(Jp[j][0], Jp[j][1], Jp[j][2], T.K[j][0], T.K[j][1],
                                      T.K[j][2]);
  return VIO_TRACK_OK;
}

// Warp state: translation (level coords, anchor form), angle and its cos/sin.
struct Warp {
  Pos t;
  float th, cs, sn;
};

// cos, sin, sin(phi)/phi and (1 - cos(phi))/phi of a small angle
__device__ __forceinline__ void small_rot(float p, float& c, float& s, float& a, float& b) {
  if (fabsf(p) < 0.25f) {
    const float p2 = __fmul_rn(p, p);
    c = __fmaf_rn(-p2, __fmaf_rn(-p2, __fmaf_rn(-p2, 1.f / 720.f, 1.f / 24.f), 0.5f), 1.f);
    a = __fmaf_rn(-p2, __fmaf_rn(-p2, __fmaf_rn(-p2, 1.f / 5040.f, 1.f / 120.f), 1.f / 6.f),
                  1.f);
    s = __fmul_rn(p, a);
    b = __fmul_rn(p, __fmaf_rn(-p2,
                               __fmaf_rn(-p2, __fmaf_rn(-p2, 1.f / 40320.f, 1.f / 720.f),
                                         1.f / 24.f),
                               0.5f));
  } else {
    sincosf(p, &s, &c);
    a = s / p;
    const float h = sinf(0.5f * p);
    b = 2.f * h * h / p;
  }
}

// 1.5 * 2^23 and its bit pattern: v + kFloorBias rounded toward -inf is
// kFloorBias + floor(v) on the integer grid of [2^23, 2^24).
constexpr float kFloorBias = 12582912.f;
constexpr int kFloorBiasBits = 0x4B400000;

// Radius of the pattern's outermost point (7, 3): an increment (dx, dy, dth)
// moves no pattern point by more than |dx| + |dy| + kPatRadius |dth| px.
constexpr float kPatRadius = 7.6158f;

// One Gauss-Newton step (Eq. 4-5). Returns a VIO_TRACK_* status; `moved` is
// the bound above on how far the step moved the pattern (level px).
template <bool BUTTERFLY = false>
__device__ __forceinline__ int gn_step(const Lv& L, const Tpl& T, int lane, const LanePts& P,
                                       Warp& W, float& moved) {
  float r0 = 0.f, r1 = 0.f, r2 = 0.f, r3 = 0.f;
  bool ok = true;
  const unsigned xmax = (unsigned)(L.w - 2), ymax = (unsigned)(L.h - 2);
  // no branch in the loop: a lane without a second point evaluates the
  // pattern's centre with weight 0 (its K is 0 too); it lies inside the
  // level whenever the pattern's points do. A sample outside the level is
  // read at the clamped position and only clears `ok`.
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    const float u = P.u[j], v = P.v[j];
    const float vx = __fmaf_rn(W.cs, u, __fmaf_rn(-W.sn, v, W.t.dx));
    const float vy = __fmaf_rn(W.sn, u, __fmaf_rn(W.cs, v, W.t.dy));
    // floor without a conversion instruction: adding 1.5 * 2^23 rounded
    // down leaves floor(v) in the low mantissa bits (exact for |v| < 2^22;
    // beyond that the sample is outside the level either way)
    const float tx = __fadd_rd(vx, kFloorBias), ty = __fadd_rd(vy, kFloorBias);
    const int ix = W.t.ax + (__float_as_int(tx) - kFloorBiasBits);
    const int iy = W.t.ay + (__float_as_int(ty) - kFloorBiasBits);
    const float fx = vx - (tx - kFloorBias), fy = vy - (ty - kFloorBias);
    // 0 <= y < w - 1 on the integer part: 0 <= ix <= w - 2 (one unsigned test)
    ok = ok && (unsigned)ix <= xmax && (unsigned)iy <= ymax;
    const unsigned cx = min((unsigned)ix, xmax), cy = min((unsigned)iy, ymax);
    const uint8_t* p = L.p + (cy * (unsigned)L.pitch + cx);
    const float a = __ldg(p), b = __ldg(p + 1);
    const float c = __ldg(p + L.pitch), d = __ldg(p + L.pitch + 1);
    const float top = __fmaf_rn(fx, b - a, a), bot = __fmaf_rn(fx, d - c, c);
    const float r = __fmaf_rn(fy, bot - top, top);
    r0 = j == 0 ? r0 + r : __fmaf_rn(P.w1, r, r0);
    r1 = __fmaf_rn(T.K[j][0], r, r1);
    r2 = __fmaf_rn(T.K[j][1], r, r2);
    r3 = __fmaf_rn(T.K[j][2], r, r3);
  }
  // a sample outside the level adds 1e30 to the sum of intensities (at most
  // 52 x 255 otherwise), so the one reduction also tells every lane whether
  // any lane left the level
  if (!ok) r0 += 1e30f;
  warp_sum4<BUTTERFLY>(r0, r1, r2, r3);
  // the increment before its checks, so that one branch takes all three
  // failures (in this order): a sample outside the level, a non-positive
  // mean, a non-finite increment (a NaN or an infinity in any component
  // fails the finite comparison)
  const float q = __fdividef(T.S, r0);
  const float d0 = __fmaf_rn(-q, r1, T.c0);
  const float d1 = __fmaf_rn(-q, r2, T.c1);
  const float d2 = __fmaf_rn(-q, r3, T.c2);
  const float s01 = fabsf(d0) + fabsf(d1);
  if (!(r0 < 1e29f && r0 > 0.f && s01 + fabsf(d2) < 3.0e38f))
    return r0 >= 1e29f ? VIO_TRACK_OOB_WARP : !(r0 > 0.f) ? VIO_TRACK_ZERO_MEAN : VIO_TRACK_NAN;
  moved = __fmaf_rn(kPatRadius, fabsf(d2), s01);
  // T <- T o exp(delta): t += R V(d2) (d0, d1), R <- R R(d2)
  float cd, sd, a, b;
  small_rot(d2, cd, sd, a, b);
  const float vx = __fmaf_rn(-b, d1, __fmul_rn(a, d0));
  const float vy = __fmaf_rn(a, d1, __fmul_rn(b, d0));
  W.t.dx = __fmaf_rn(W.cs, vx, __fmaf_rn(-W.sn, vy, W.t.dx));
  W.t.dy = __fmaf_rn(W.sn, vx, __fmaf_rn(W.cs, vy, W.t.dy));
  const float cs = __fmaf_rn(-W.sn, sd, __fmul_rn(W.cs, cd));
  const float sn = __fmaf_rn(W.cs, sd, __fmul_rn(W.sn, cd));
  W.cs = cs;
  W.sn = sn;
  W.th += d2;
  return VIO_TRACK_OK;
}

__device__ __forceinline__ Lv get_lv(const Geom& g, const Batch& b, int img, int l) {
  return Lv{level_ptr(g, b, img, l), g.w[l], g.h[l], g.pitch[l]};
}

// Coarse-to-fine tracking of keypoint p (anchor form) of image src_img of the
// source batch into image dst_img of the target batch, from warp (t0, th0) at
// level 0, over levels top..0 (top = n_levels - 1 is the whole pyramid). A
// level whose template is invalid is skipped, except level 0; any warp
// failure ends the track. last_step: how far the last Gauss-Newton step at
// level 0 moved the pattern (bound of gn_step, level-0 px; 0 if none ran).
template <bool BUTTERFLY = false>
__device__ __forceinline__ int track_dir(const Geom& g, const Batch& src, int src_img,
                                         const Batch& dst, int dst_img, const Pos& p, Pos t0,
                                         float th0, int iters, int top, int lane, Pos& t_out,
                                         float& th_out, float& last_step) {
  Warp W;
  last_step = 0.f;
  to_level1(t0.ax, t0.dx, top, W.t.ax, W.t.dx);
  to_level1(t0.ay, t0.dy, top, W.t.ay, W.t.dy);
  W.th = th0;
  {
    float a, b;
    small_rot(th0, W.cs, W.sn, a, b);
  }
  const LanePts P = lane_points(lane);
  Tpl T;
  for (int l = top; l >= 0; --l) {
    const int ts = build_template(get_lv(g, src, src_img, l), p, l, lane, P, T);
    if (ts != VIO_TRACK_OK) {
      if (l == 0) return ts;
    } else {
      const Lv D = get_lv(g, dst, dst_img, l);
      float moved = 0.f;
      for (int it = 0; it < iters; ++it) {
        const int st = gn_step<BUTTERFLY>(D, T, lane, P, W, moved);
        if (st != VIO_TRACK_OK) return st;
      }
      if (l == 0) last_step = moved;
      rebase(W.t);
    }
    if (l > 0) {
      W.t.ax *= 2;
      W.t.ay *= 2;
      W.t.dx *= 2.f;
      W.t.dy *= 2.f;
      rebase(W.t);
    }
  }
  t_out = W.t;
  th_out = W.th;
  return VIO_TRACK_OK;
}

// Forward track with the optional backward pass and distance check, both
// over levels top..0, from warp (ix, iy, ith) if has_init, else from p.
// Returns the status; tf/thf hold the forward result when it exists and
// last_fwd the forward pass's last level-0 step (track_dir).
template <bool BUTTERFLY = false>
__device__ __forceinline__ int track_fb(const Geom& g, const Batch& src, int src_img,
                                        const Batch& dst, int dst_img, float px, float py,
                                        bool has_init, float ix, float iy, float ith,
                                        const TrackCfg& cfg, int top, int lane, Pos& tf,
                                        float& thf, bool& have, float& dist, float& last_fwd) {
  const Pos p = split(px, py);
  Pos t0 = p;
  float th0 = 0.f;
  if (has_init) {
    t0 = split(ix, iy);
    th0 = ith;
  }
  int st = track_dir<BUTTERFLY>(g, src, src_img, dst, dst_img, p, t0, th0, cfg.gn_iters, top,
                                lane, tf, thf, last_fwd);
  have = st == VIO_TRACK_OK;
  dist = __int_as_float(0x7fc00000);
  if (st == VIO_TRACK_OK && cfg.fb) {
    // backward: template on the target at the forward result, unrotated;
    // start at the forward estimate's inverse (t = p, theta = -theta_f)
    Pos tb;
    float thb, last_b;
    st = track_dir<BUTTERFLY>(g, dst, dst_img, src, src_img, tf, p, -thf, cfg.gn_iters, top,
                              lane, tb, thb, last_b);
    if (st == VIO_TRACK_OK) {
      const float ex = (float)(tb.ax - p.ax) + (tb.dx - p.dx);
      const float ey = (float)(tb.ay - p.ay) + (tb.dy - p.dy);
      dist = sqrtf(__fmaf_rn(ey, ey, __fmul_rn(ex, ex)));
      if (dist > cfg.fb_max_dist) st = VIO_TRACK_FB_FAIL;
    }
  }
  return st;
}

}  // namespace trk
}  // namespace vio
