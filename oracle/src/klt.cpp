/*
 * CPU oracle: patch-based inverse-compositional KLT with an SE(2) warp,
 * pyramidal, with a forward-backward check (Sec. III-E, Eq. 4-5).
 * TEST INFRASTRUCTURE ONLY; see oracle.h. FP64 throughout.
 */
#include "oracle.h"

#include <cmath>
#include <limits>
#include <thread>
#include <vector>

namespace {

constexpr int kMaxPts = 64;

/* Sec. III-E fixes only the count of the sample pattern (52 points). This
 * oracle's reading: the odd lattice u, v in {+-1, +-3, +-5, +-7} with
 * |u| + |v| <= 10, i.e. the 8x8 lattice at 2 px spacing minus the three
 * outermost points of each corner; ordered by v, then u. */
int pattern_points(int pattern_id, double* u, double* v) {
  if (pattern_id != 0) return 0;
  int n = 0;
  for (int iv = -7; iv <= 7; iv += 2)
    for (int iu = -7; iu <= 7; iu += 2)
      if (std::abs(iu) + std::abs(iv) <= 10) {
        u[n] = iu;
        v[n] = iv;
        ++n;
      }
  return n;
}

/* Records min |value - bound| (scaled to level-0 px) and tests lo <= v < hi. */
inline bool in_bounds(double val, double lo, double hi, double scale, double* margin) {
  if (margin) {
    const double m = std::min(std::fabs(val - lo), std::fabs(hi - val)) * scale;
    if (m < *margin) *margin = m;
  }
  return val >= lo && val < hi;
}

/* Bilinear interpolation of a uint8 plane with pixel centres at integer
 * coordinates. Needs 0 <= x < w-1 and 0 <= y < h-1 (checked by callers). */
double bilinear(const vo_image& im, double x, double y) {
  const double fx0 = std::floor(x), fy0 = std::floor(y);
  const int x0 = (int)fx0, y0 = (int)fy0;
  const double ax = x - fx0, ay = y - fy0;
  const uint8_t* r0 = im.data + (long)y0 * im.pitch + x0;
  const uint8_t* r1 = r0 + im.pitch;
  return (1 - ax) * (1 - ay) * r0[0] + ax * (1 - ay) * r0[1] + (1 - ax) * ay * r1[0] +
         ax * ay * r1[1];
}

struct Template {
  int np;
  double u[kMaxPts], v[kMaxPts];
  double s[kMaxPts];           /* raw samples                               */
  double gx[kMaxPts], gy[kMaxPts];
  double mean;                 /* I-bar of Eq. 4                           */
  double sn[kMaxPts];          /* mean-normalised samples                  */
  double J[kMaxPts][3];        /* rows J_i of the normalised patch         */
  double H[3][3];              /* J^T J                                    */
  double G[3][kMaxPts];        /* H^-1 J^T                                 */
};

/* Solve H x = b for symmetric positive definite 3x3 H by Cholesky. Returns
 * false if a pivot is <= 1e-9 * trace(H) (the oracle's degeneracy rule; the
 * paper does not give one). */
bool chol3(const double H[3][3], double L[3][3]) {
  const double tr = H[0][0] + H[1][1] + H[2][2];
  const double eps = 1e-9 * tr;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) L[i][j] = 0;
  for (int j = 0; j < 3; ++j) {
    double d = H[j][j];
    for (int k = 0; k < j; ++k) d -= L[j][k] * L[j][k];
    if (!(d > eps)) return false;
    L[j][j] = std::sqrt(d);
    for (int i = j + 1; i < 3; ++i) {
      double s = H[i][j];
      for (int k = 0; k < j; ++k) s -= L[i][k] * L[j][k];
      L[i][j] = s / L[j][j];
    }
  }
  return true;
}

void chol3_solve(const double L[3][3], const double b[3], double x[3]) {
  double y[3];
  for (int i = 0; i < 3; ++i) {
    double s = b[i];
    for (int k = 0; k < i; ++k) s -= L[i][k] * y[k];
    y[i] = s / L[i][i];
  }
  for (int i = 2; i >= 0; --i) {
    double s = y[i];
    for (int k = i + 1; k < 3; ++k) s -= L[k][i] * x[k];
    x[i] = s / L[i][i];
  }
}

/* Sec. III-E: the template of a keypoint q at one level, from the source
 * image. Samples s_i = I(q + x_i); the gradient (g_x, g_y) is the central
 * difference of the bilinear interpolant one pixel either side (the paper
 * names the gradient but not its operator). Eq. 4 divides the patch by its
 * mean, so the template is s_i / I-bar with gradient g_i / I-bar. Then
 * J_i = [g_x, g_y, g_y u_i - g_x v_i], H = J^T J and G = H^-1 J^T. */
int build_template(const vo_image& im, double qx, double qy, int pattern_id, double scale,
                   Template& T, double* margin) {
  T.np = pattern_points(pattern_id, T.u, T.v);
  if (T.np == 0) return VO_OOB_TEMPLATE;
  for (int i = 0; i < T.np; ++i) {
    const double cx = qx + T.u[i], cy = qy + T.v[i];
    /* bilinear at c +- 1 needs 0 <= c-1 and c+1 < w-1 */
    const bool okx = in_bounds(cx, 1.0, (double)im.w - 2.0, scale, margin);
    const bool oky = in_bounds(cy, 1.0, (double)im.h - 2.0, scale, margin);
    if (!okx || !oky) return VO_OOB_TEMPLATE;
  }
  double sum = 0;
  for (int i = 0; i < T.np; ++i) {
    const double cx = qx + T.u[i], cy = qy + T.v[i];
    T.s[i] = bilinear(im, cx, cy);
    T.gx[i] = 0.5 * (bilinear(im, cx + 1, cy) - bilinear(im, cx - 1, cy));
    T.gy[i] = 0.5 * (bilinear(im, cx, cy + 1) - bilinear(im, cx, cy - 1));
    sum += T.s[i];
  }
  T.mean = sum / T.np;
  if (!(T.mean > 0)) return VO_ZERO_MEAN;
  for (int i = 0; i < T.np; ++i) {
    T.sn[i] = T.s[i] / T.mean;
    const double gx = T.gx[i] / T.mean, gy = T.gy[i] / T.mean;
    T.J[i][0] = gx;
    T.J[i][1] = gy;
    T.J[i][2] = gy * T.u[i] - gx * T.v[i];
  }
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      double h = 0;
      for (int i = 0; i < T.np; ++i) h += T.J[i][a] * T.J[i][b];
      T.H[a][b] = h;
    }
  double L[3][3];
  if (!chol3(T.H, L)) return VO_DEGENERATE_H;
  for (int i = 0; i < T.np; ++i) {
    double g[3];
    chol3_solve(L, T.J[i], g);
    for (int a = 0; a < 3; ++a) T.G[a][i] = g[a];
  }
  return VO_OK;
}

/* SE(2) exponential: exp(dx, dy, dth) = (R(dth), V(dth) (dx, dy)) with
 * V(phi) = [[sin phi/phi, -(1-cos phi)/phi], [(1-cos phi)/phi, sin phi/phi]]. */
void se2_exp(double dx, double dy, double dth, double R[2][2], double t[2]) {
  const double c = std::cos(dth), s = std::sin(dth);
  double a, b; /* sin(phi)/phi, (1-cos(phi))/phi */
  if (std::fabs(dth) < 1e-9) {
    a = 1.0 - dth * dth / 6.0;
    b = 0.5 * dth;
  } else {
    a = s / dth;
    b = (1.0 - c) / dth;
  }
  R[0][0] = c;
  R[0][1] = -s;
  R[1][0] = s;
  R[1][1] = c;
  t[0] = a * dx - b * dy;
  t[1] = b * dx + a * dy;
}

struct Warp {
  double tx, ty, th; /* target position of the keypoint (current level), angle */
};

/* One Gauss-Newton step (Eq. 4-5) at one level. The warp maps pattern offset
 * x_i to R(theta) x_i + t in the target image. *moved receives
 * |dx| + |dy| + r |dtheta| of the increment, r the pattern's largest radius:
 * a bound on how far the step moved any pattern point (level px), the
 * convergence measure of the learned start's gate. */
int gn_step(const vo_image& tgt, const Template& T, double scale, Warp& W, double* margin,
            double* moved) {
  const double c = std::cos(W.th), s = std::sin(W.th);
  double r[kMaxPts];
  double sum = 0;
  for (int i = 0; i < T.np; ++i) {
    const double yx = c * T.u[i] - s * T.v[i] + W.tx;
    const double yy = s * T.u[i] + c * T.v[i] + W.ty;
    const bool okx = in_bounds(yx, 0.0, (double)tgt.w - 1.0, scale, margin);
    const bool oky = in_bounds(yy, 0.0, (double)tgt.h - 1.0, scale, margin);
    if (!okx || !oky) return VO_OOB_WARP;
    r[i] = bilinear(tgt, yx, yy);
    sum += r[i];
  }
  const double rmean = sum / T.np;
  if (!(rmean > 0)) return VO_ZERO_MEAN;
  /* Eq. 4: e_i = I_{t+1}(T x_i) / mean_{t+1} - I_t(x_i) / mean_t */
  double e[kMaxPts];
  for (int i = 0; i < T.np; ++i) e[i] = r[i] / rmean - T.sn[i];
  /* Eq. 5: delta = -G e, T <- T o exp(delta) */
  double d[3];
  for (int a = 0; a < 3; ++a) {
    double acc = 0;
    for (int i = 0; i < T.np; ++i) acc += T.G[a][i] * e[i];
    d[a] = -acc;
  }
  if (!std::isfinite(d[0]) || !std::isfinite(d[1]) || !std::isfinite(d[2])) return VO_NAN;
  double rmax = 0;
  for (int i = 0; i < T.np; ++i) rmax = std::max(rmax, std::hypot(T.u[i], T.v[i]));
  *moved = std::fabs(d[0]) + std::fabs(d[1]) + rmax * std::fabs(d[2]);
  double Rd[2][2], td[2];
  se2_exp(d[0], d[1], d[2], Rd, td);
  /* (R, t) o (Rd, td) = (R Rd, R td + t); R Rd is the rotation by th + dth */
  W.tx += c * td[0] - s * td[1];
  W.ty += s * td[0] + c * td[1];
  W.th += d[2];
  return VO_OK;
}

/* Pyramidal tracking of one keypoint p from src to dst, coarse to fine
 * (Sec. III-E). The template is rebuilt at every level from the source; a
 * level whose template is invalid is skipped except at level 0, where its
 * status ends the track (the paper does not say how such levels are
 * handled). Any warp failure ends the track at once. */
int track_one(const vo_pyramid& src, const vo_pyramid& dst, int n_levels, double px,
              double py, const Warp& init, const vo_track_params& prm, Warp& out,
              double* margin, double* last_step) {
  Warp W = init;
  *last_step = 0;
  const double top = std::ldexp(1.0, n_levels - 1);
  W.tx /= top;
  W.ty /= top;
  Template T;
  for (int l = n_levels - 1; l >= 0; --l) {
    const double scale = std::ldexp(1.0, l);
    const int ts = build_template(src.lv[l], px / scale, py / scale, prm.pattern_id, scale, T,
                                  margin);
    if (ts != VO_OK) {
      if (l == 0) return ts;
    } else {
      double moved = 0;
      for (int it = 0; it < prm.gn_iters; ++it) {
        const int st = gn_step(dst.lv[l], T, scale, W, margin, &moved);
        if (st != VO_OK) return st;
      }
      if (l == 0) *last_step = moved;
    }
    if (l > 0) {
      W.tx *= 2;
      W.ty *= 2;
    }
  }
  out = W;
  return VO_OK;
}

void track_range(const vo_pyramid* src, const vo_pyramid* dst, int i0, int i1, const float* pts,
                 const float* init, const vo_track_params* p, int fb, double* warp,
                 uint8_t* status, double* fb_dist, double* margin, double* back,
                 double* last_step) {
  const int L = std::min(src->n_levels, dst->n_levels);
  const double nan = std::numeric_limits<double>::quiet_NaN();
  for (int i = i0; i < i1; ++i) {
    const double px = pts[2 * i], py = pts[2 * i + 1];
    Warp w0{px, py, 0.0};
    if (init) w0 = Warp{init[3 * i], init[3 * i + 1], init[3 * i + 2]};
    double m = std::numeric_limits<double>::infinity();
    Warp wf{nan, nan, nan}, wb{nan, nan, nan};
    double last = nan, last_b = nan;
    int st = track_one(*src, *dst, L, px, py, w0, *p, wf, &m, &last);
    if (st != VO_OK) last = nan;
    double dist = nan;
    if (st == VO_OK && fb) {
      /* Backward pass (Sec. III-E): the template is rebuilt on the target
       * image at the forward result, unrotated, and the warp starts from the
       * forward estimate's inverse, which in this parametrisation is the
       * original position p with angle -theta_f. */
      const Warp wbi{px, py, -wf.th};
      st = track_one(*dst, *src, L, wf.tx, wf.ty, wbi, *p, wb, &m, &last_b);
      if (st == VO_OK) {
        dist = std::hypot(wb.tx - px, wb.ty - py);
        if (dist > p->fb_max_dist) st = VO_FB_FAIL;
      }
    }
    status[i] = (uint8_t)st;
    warp[3 * i] = wf.tx;
    warp[3 * i + 1] = wf.ty;
    warp[3 * i + 2] = wf.th;
    if (fb_dist) fb_dist[i] = dist;
    if (margin) margin[i] = m;
    if (last_step) last_step[i] = last;
    if (back) {
      back[3 * i] = wb.tx;
      back[3 * i + 1] = wb.ty;
      back[3 * i + 2] = wb.th;
    }
  }
}

}  // namespace

extern "C" int32_t vo_pattern(int32_t pattern_id, double* u, double* v) {
  return pattern_points(pattern_id, u, v);
}

extern "C" void vo_se2_exp(double dx, double dy, double dth, double* M) {
  double R[2][2], t[2];
  se2_exp(dx, dy, dth, R, t);
  M[0] = R[0][0];
  M[1] = R[0][1];
  M[2] = t[0];
  M[3] = R[1][0];
  M[4] = R[1][1];
  M[5] = t[1];
  M[6] = 0;
  M[7] = 0;
  M[8] = 1;
}

extern "C" int32_t vo_template(const vo_image* img, double qx, double qy, int32_t pattern_id,
                               double* s, double* gx, double* gy, double* J, double* H,
                               double* G, double* mean) {
  Template T;
  const int st = build_template(*img, qx, qy, pattern_id, 1.0, T, nullptr);
  if (st == VO_OOB_TEMPLATE) return st;
  for (int i = 0; i < T.np; ++i) {
    s[i] = T.s[i];
    gx[i] = T.gx[i];
    gy[i] = T.gy[i];
  }
  *mean = T.mean;
  if (st != VO_OK && st != VO_DEGENERATE_H) return st;
  for (int i = 0; i < T.np; ++i)
    for (int a = 0; a < 3; ++a) J[3 * i + a] = T.J[i][a];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) H[3 * a + b] = T.H[a][b];
  if (st == VO_OK)
    for (int a = 0; a < 3; ++a)
      for (int i = 0; i < T.np; ++i) G[a * T.np + i] = T.G[a][i];
  return st;
}

extern "C" void vo_track(const vo_pyramid* src, const vo_pyramid* dst, int32_t n,
                         const float* pts, const float* init, const vo_track_params* p,
                         int32_t fb, double* warp, uint8_t* status, double* fb_dist,
                         double* margin, double* back, double* last_step, int32_t n_threads) {
  if (n_threads <= 1 || n < 64) {
    track_range(src, dst, 0, n, pts, init, p, fb, warp, status, fb_dist, margin, back,
                last_step);
    return;
  }
  std::vector<std::thread> pool;
  const int per = (n + n_threads - 1) / n_threads;
  for (int t = 0; t < n_threads; ++t) {
    const int i0 = t * per, i1 = std::min(n, i0 + per);
    if (i0 >= i1) break;
    pool.emplace_back(track_range, src, dst, i0, i1, pts, init, p, fb, warp, status, fb_dist,
                      margin, back, last_step);
  }
  for (auto& th : pool) th.join();
}
