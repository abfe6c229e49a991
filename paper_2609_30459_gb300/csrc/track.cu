// Pyramidal inverse-compositional KLT with an SE(2) warp (Sec. III-E,
// Eq. 4-5), one warp of 32 threads per keypoint; each lane owns up to two of
// the 52 pattern points and the warp combines its sums with xor shuffles.
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
// Positions keep an integer anchor plus a small float offset, so that bilinear
// weights carry full FP32 precision at any image size; template samples of
// one keypoint share one sub-pixel offset and therefore one set of weights.
#include <math.h>

#include "common.cuh"

namespace vio {
namespace {

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
__constant__ Pattern kPat = make_pattern();
static_assert(make_pattern().n == 52, "pattern size");
constexpr int kNP = 52;

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

__device__ __forceinline__ float bilerp(float a, float b, float c, float d, float w00, float w10,
                                        float w01, float w11) {
  return w00 * a + w10 * b + w01 * c + w11 * d;
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

// anchor + offset scaled to level l: (a + d) / 2^l as anchor + offset in [0,1)
__device__ __forceinline__ void to_level(const Pos& p0, int l, int& Q, float& f, bool y) {
  const int a = y ? p0.ay : p0.ax;
  const float d = y ? p0.dy : p0.dx;
  const int Ql = a >> l;
  const float frac = ((float)(a - Ql * (1 << l)) + d) * __int_as_float((127 - l) << 23);
  const float fl = floorf(frac);
  Q = Ql + (int)fl;
  f = frac - fl;
}

struct Tpl {
  float K[2][3];   // H'^-1 J'_i for the lane's two points
  float c[3];      // H'^-1 sum J'_i s_i
  float S;         // sum s_i
};

// Builds the template of keypoint q (level-0 anchor form) at level l of the
// source. Returns a VIO_TRACK_* status (uniform across the warp).
__device__ int build_template(const Lv& L, const Pos& q, int l, int lane, Tpl& T) {
  int Qx, Qy;
  float fx, fy;
  to_level(q, l, Qx, fx, false);
  to_level(q, l, Qy, fy, true);
  // bilinear at c and c +- 1 needs 1 <= c < w - 2: on integers, 1 <= Q + u <= w - 3
  bool ok = true;
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    const int i = lane + 32 * j;
    if (i < kNP) {
      const int ix = Qx + kPat.u[i], iy = Qy + kPat.v[i];
      ok = ok && ix >= 1 && ix <= L.w - 3 && iy >= 1 && iy <= L.h - 3;
    }
  }
  if (!__all_sync(0xffffffffu, ok)) return VIO_TRACK_OOB_TEMPLATE;

  const float w00 = (1.f - fx) * (1.f - fy), w10 = fx * (1.f - fy);
  const float w01 = (1.f - fx) * fy, w11 = fx * fy;
  float Jp[2][3], sv[2];
  float acc[10];
#pragma unroll
  for (int i = 0; i < 10; ++i) acc[i] = 0.f;
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    const int i = lane + 32 * j;
    Jp[j][0] = Jp[j][1] = Jp[j][2] = 0.f;
    sv[j] = 0.f;
    if (i < kNP) {
      const float u = kPat.u[i], v = kPat.v[i];
      const uint8_t* base = L.p + (long long)(Qy + kPat.v[i] - 1) * L.pitch + (Qx + kPat.u[i] - 1);
      float t[4][4];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int cc = 0; cc < 4; ++cc)
          t[r][cc] = (r == 0 || r == 3) && (cc == 0 || cc == 3)
                         ? 0.f
                         : (float)__ldg(base + (long long)r * L.pitch + cc);
      const float s = bilerp(t[1][1], t[1][2], t[2][1], t[2][2], w00, w10, w01, w11);
      const float bxp = bilerp(t[1][2], t[1][3], t[2][2], t[2][3], w00, w10, w01, w11);
      const float bxm = bilerp(t[1][0], t[1][1], t[2][0], t[2][1], w00, w10, w01, w11);
      const float byp = bilerp(t[2][1], t[2][2], t[3][1], t[3][2], w00, w10, w01, w11);
      const float bym = bilerp(t[0][1], t[0][2], t[1][1], t[1][2], w00, w10, w01, w11);
      const float gx = 0.5f * (bxp - bxm), gy = 0.5f * (byp - bym);
      Jp[j][0] = gx;
      Jp[j][1] = gy;
      Jp[j][2] = gy * u - gx * v;
      sv[j] = s;
      acc[0] += s;
      acc[1] += Jp[j][0] * Jp[j][0];
      acc[2] += Jp[j][0] * Jp[j][1];
      acc[3] += Jp[j][0] * Jp[j][2];
      acc[4] += Jp[j][1] * Jp[j][1];
      acc[5] += Jp[j][1] * Jp[j][2];
      acc[6] += Jp[j][2] * Jp[j][2];
      acc[7] += Jp[j][0] * s;
      acc[8] += Jp[j][1] * s;
      acc[9] += Jp[j][2] * s;
    }
  }
  warp_sum(acc);
  T.S = acc[0];
  if (!(acc[0] > 0.f)) return VIO_TRACK_ZERO_MEAN;
  // Cholesky of H'; a pivot <= 1e-9 trace marks a degenerate patch
  const float h00 = acc[1], h01 = acc[2], h02 = acc[3], h11 = acc[4], h12 = acc[5],
              h22 = acc[6];
  const float eps = 1e-9f * (h00 + h11 + h22);
  if (!(h00 > eps)) return VIO_TRACK_DEGENERATE_H;
  const float l00 = sqrtf(h00);
  const float l10 = h01 / l00, l20 = h02 / l00;
  const float d1 = h11 - l10 * l10;
  if (!(d1 > eps)) return VIO_TRACK_DEGENERATE_H;
  const float l11 = sqrtf(d1);
  const float l21 = (h12 - l20 * l10) / l11;
  const float d2 = h22 - l20 * l20 - l21 * l21;
  if (!(d2 > eps)) return VIO_TRACK_DEGENERATE_H;
  const float l22 = sqrtf(d2);
  auto solve = [&](const float b0, const float b1, const float b2, float* x) {
    const float y0 = b0 / l00;
    const float y1 = (b1 - l10 * y0) / l11;
    const float y2 = (b2 - l20 * y0 - l21 * y1) / l22;
    x[2] = y2 / l22;
    x[1] = (y1 - l21 * x[2]) / l11;
    x[0] = (y0 - l10 * x[1] - l20 * x[2]) / l00;
  };
  solve(acc[7], acc[8], acc[9], T.c);
#pragma unroll
  for (int j = 0; j < 2; ++j) solve(Jp[j][0], Jp[j][1], Jp[j][2], T.K[j]);
  return VIO_TRACK_OK;
}

// One Gauss-Newton step (Eq. 4-5). Warp: rotation th, translation t (level
// coords, anchor form). Returns a VIO_TRACK_* status.
__device__ int gn_step(const Lv& L, const Tpl& T, int lane, Pos& t, float& th) {
  float sn, cs;
  sincosf(th, &sn, &cs);
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
  bool ok = true;
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    const int i = lane + 32 * j;
    if (i < kNP) {
      const float u = kPat.u[i], v = kPat.v[i];
      const float vx = cs * u - sn * v + t.dx;
      const float vy = sn * u + cs * v + t.dy;
      const float flx = floorf(vx), fly = floorf(vy);
      const int ix = t.ax + (int)flx, iy = t.ay + (int)fly;
      const float fx = vx - flx, fy = vy - fly;
      // 0 <= y < w - 1 on the integer part: 0 <= ix <= w - 2
      if (ix >= 0 && ix <= L.w - 2 && iy >= 0 && iy <= L.h - 2) {
        const uint8_t* p = L.p + (long long)iy * L.pitch + ix;
        const float a = __ldg(p), b = __ldg(p + 1);
        const float c = __ldg(p + L.pitch), d = __ldg(p + L.pitch + 1);
        const float r = (1.f - fx) * (1.f - fy) * a + fx * (1.f - fy) * b +
                        (1.f - fx) * fy * c + fx * fy * d;
        acc[0] += r;
        acc[1] += T.K[j][0] * r;
        acc[2] += T.K[j][1] * r;
        acc[3] += T.K[j][2] * r;
      } else {
        ok = false;
      }
    }
  }
  if (!__all_sync(0xffffffffu, ok)) return VIO_TRACK_OOB_WARP;
  warp_sum(acc);
  if (!(acc[0] > 0.f)) return VIO_TRACK_ZERO_MEAN;
  const float q = T.S / acc[0];
  const float d0 = T.c[0] - q * acc[1];
  const float d1 = T.c[1] - q * acc[2];
  const float d2 = T.c[2] - q * acc[3];
  if (!isfinite(d0) || !isfinite(d1) || !isfinite(d2)) return VIO_TRACK_NAN;
  // T <- T o exp(delta): t += R(th) V(d2) (d0, d1), th += d2, with
  // V = [[a, -b], [b, a]], a = sin(phi)/phi, b = (1 - cos(phi))/phi = 2 sin^2(phi/2)/phi
  float a = 1.f, b = 0.f;
  if (d2 != 0.f) {
    const float sh = sinf(0.5f * d2);
    a = sinf(d2) / d2;
    b = 2.f * sh * sh / d2;
  }
  const float vx = a * d0 - b * d1, vy = b * d0 + a * d1;
  t.dx += cs * vx - sn * vy;
  t.dy += sn * vx + cs * vy;
  th += d2;
  rebase(t);
  return VIO_TRACK_OK;
}

__device__ __forceinline__ Lv get_lv(const Geom& g, const Batch& b, int img, int l) {
  return Lv{level_ptr(g, b, img, l), g.w[l], g.h[l], g.pitch[l]};
}

// Coarse-to-fine tracking of keypoint p (anchor form) from src to dst,
// starting from warp (t0, th0) at level 0. A level whose template is invalid
// is skipped, except level 0; any warp failure ends the track.
__device__ int track_dir(const Geom& g, const Batch& src, const Batch& dst, int img,
                         const Pos& p, Pos t0, float th0, int iters, int lane, Pos& t_out,
                         float& th_out) {
  const int L = g.n_levels;
  // start at the top level: t0 / 2^(L-1)
  Pos t;
  {
    int Q;
    float f;
    to_level(t0, L - 1, Q, f, false);
    t.ax = Q;
    t.dx = f;
    to_level(t0, L - 1, Q, f, true);
    t.ay = Q;
    t.dy = f;
  }
  float th = th0;
  Tpl T;
  for (int l = L - 1; l >= 0; --l) {
    const int ts = build_template(get_lv(g, src, img, l), p, l, lane, T);
    if (ts != VIO_TRACK_OK) {
      if (l == 0) return ts;
    } else {
      const Lv D = get_lv(g, dst, img, l);
      for (int it = 0; it < iters; ++it) {
        const int st = gn_step(D, T, lane, t, th);
        if (st != VIO_TRACK_OK) return st;
      }
    }
    if (l > 0) {
      t.ax *= 2;
      t.ay *= 2;
      t.dx *= 2.f;
      t.dy *= 2.f;
      rebase(t);
    }
  }
  t_out = t;
  th_out = th;
  return VIO_TRACK_OK;
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

struct TrackArgs {
  Geom g;
  Batch src, dst;
  const float* pts;    // float2 per slot
  const float* init;   // float3 per slot or null
  const int32_t* count;
  int capacity, n_images;
  TrackCfg cfg;
  float* out3;         // float3 per slot or null
  float* out2;         // float2 per slot or null
  uint8_t* status;
  float* fb_dist;
};

constexpr int TRK_THREADS = 128;

__global__ void __launch_bounds__(TRK_THREADS) track_kernel(TrackArgs a) {
  const long long wid = ((long long)blockIdx.x * TRK_THREADS + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const long long total = (long long)a.capacity * a.n_images;
  if (wid >= total) return;
  const int img = (int)(wid / a.capacity);
  const int k = (int)(wid - (long long)img * a.capacity);
  const int n = a.count ? min(a.count[img], a.capacity) : a.capacity;
  const float nanf_ = __int_as_float(0x7fc00000);
  if (k >= n) {
    if (lane == 0) {
      a.status[wid] = VIO_TRACK_EMPTY;
      if (a.out3) a.out3[3 * wid] = a.out3[3 * wid + 1] = a.out3[3 * wid + 2] = nanf_;
      if (a.out2) a.out2[2 * wid] = a.out2[2 * wid + 1] = nanf_;
      if (a.fb_dist) a.fb_dist[wid] = nanf_;
    }
    return;
  }
  const float px = a.pts[2 * wid], py = a.pts[2 * wid + 1];
  const Pos p = split(px, py);
  Pos t0 = p;
  float th0 = 0.f;
  if (a.init) {
    t0 = split(a.init[3 * wid], a.init[3 * wid + 1]);
    th0 = a.init[3 * wid + 2];
  }
  Pos tf;
  float thf = 0.f;
  int st = track_dir(a.g, a.src, a.dst, img, p, t0, th0, a.cfg.gn_iters, lane, tf, thf);
  const bool have = st == VIO_TRACK_OK;   // forward result exists
  float dist = nanf_;
  if (st == VIO_TRACK_OK && a.cfg.fb) {
    // backward: template on the target at the forward result, unrotated;
    // start at the forward estimate's inverse (t = p, theta = -theta_f)
    Pos tb;
    float thb;
    st = track_dir(a.g, a.dst, a.src, img, tf, p, -thf, a.cfg.gn_iters, lane, tb, thb);
    if (st == VIO_TRACK_OK) {
      const float ex = (float)(tb.ax - p.ax) + (tb.dx - p.dx);
      const float ey = (float)(tb.ay - p.ay) + (tb.dy - p.dy);
      dist = sqrtf(ex * ex + ey * ey);
      if (dist > a.cfg.fb_max_dist) st = VIO_TRACK_FB_FAIL;
    }
  }
  if (lane == 0) {
    a.status[wid] = (uint8_t)st;
    const float ox = have ? (float)tf.ax + tf.dx : nanf_;
    const float oy = have ? (float)tf.ay + tf.dy : nanf_;
    if (a.out3) {
      a.out3[3 * wid] = ox;
      a.out3[3 * wid + 1] = oy;
      a.out3[3 * wid + 2] = have ? thf : nanf_;
    }
    if (a.out2) {
      a.out2[2 * wid] = ox;
      a.out2[2 * wid + 1] = oy;
    }
    if (a.fb_dist) a.fb_dist[wid] = dist;
  }
}

__global__ void fb_check_kernel(const float* __restrict__ orig, const float* __restrict__ back,
                                const int32_t* __restrict__ count, int capacity,
                                long long total, float max_dist, uint8_t* __restrict__ status,
                                float* __restrict__ dist) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= total) return;
  const int img = (int)(i / capacity);
  const int k = (int)(i - (long long)img * capacity);
  const int n = count ? min(count[img], capacity) : capacity;
  if (k >= n || status[i] != VIO_TRACK_OK) return;
  const float ex = back[3 * i] - orig[2 * i];
  const float ey = back[3 * i + 1] - orig[2 * i + 1];
  const float d = sqrtf(ex * ex + ey * ey);
  if (dist) dist[i] = d;
  if (!(d <= max_dist)) status[i] = VIO_TRACK_FB_FAIL;
}

}  // namespace

cudaError_t launch_track(const Geom& g, const Batch& src, const Batch& dst, const float* pts,
                         const float* init, const int32_t* count, int capacity,
                         const TrackCfg& cfg, float* out3, float* out2, uint8_t* status,
                         float* fb_dist, cudaStream_t s) {
  TrackArgs a{g, src, dst, pts, init, count, capacity, src.n, cfg, out3, out2, status, fb_dist};
  const long long warps = (long long)capacity * src.n;
  if (warps == 0) return cudaSuccess;
  const long long blocks = (warps * 32 + TRK_THREADS - 1) / TRK_THREADS;
  track_kernel<<<(unsigned)blocks, TRK_THREADS, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_fb_check(const float* orig, const float* back, const int32_t* count,
                            int capacity, int n_images, float max_dist, uint8_t* status,
                            float* dist, cudaStream_t s) {
  const long long total = (long long)capacity * n_images;
  if (total == 0) return cudaSuccess;
  fb_check_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(orig, back, count, capacity,
                                                                  total, max_dist, status, dist);
  return cudaGetLastError();
}

}  // namespace vio
