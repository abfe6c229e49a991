/*
 * CPU oracle: pyramid (Sec. III-C) and grid-cell FAST-9 detection
 * (Sec. III-D). TEST INFRASTRUCTURE ONLY; see oracle.h.
 */
#include "oracle.h"

#include <algorithm>
#include <vector>

namespace {

inline int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

inline int px(const uint8_t* img, int pitch, int x, int y) {
  return (int)img[(long)y * pitch + x];
}

}  // namespace

/* Eq. 1: L_{l+1}(x,y) = round( (1/256) sum_i sum_j w_i w_j L_l(2x+i, 2y+j) ),
 * w = [1,4,6,4,1] indexed -2..2. Written as the 2-D double sum of Eq. 1, not
 * the separable form of Eq. 2-3 (the tests check that the two agree).
 * Rounding: Eq. 1 asks for the nearest integer, Eq. 3 shifts right by 8 (a
 * floor); both are offered. Pixels outside the level are clamped to the edge
 * (the paper does not say). */
extern "C" void vo_pyr_down(const uint8_t* src, int32_t w, int32_t h, int32_t src_pitch,
                            uint8_t* dst, int32_t dst_pitch, int32_t round_mode) {
  static const int wts[5] = {1, 4, 6, 4, 1};
  const int w2 = w / 2, h2 = h / 2;
  for (int y = 0; y < h2; ++y) {
    for (int x = 0; x < w2; ++x) {
      long s = 0;
      for (int j = -2; j <= 2; ++j) {
        for (int i = -2; i <= 2; ++i) {
          const int sx = clampi(2 * x + i, 0, w - 1);
          const int sy = clampi(2 * y + j, 0, h - 1);
          s += (long)wts[i + 2] * wts[j + 2] * px(src, src_pitch, sx, sy);
        }
      }
      const long v = (round_mode == 0) ? ((s + 128) >> 8) : (s >> 8);
      dst[(long)y * dst_pitch + x] = (uint8_t)v;
    }
  }
}

/* The 16 pixels of the radius-3 Bresenham circle, clockwise from the top.
 * Indices 0, 4, 8, 12 are top, right, bottom, left: the opposite pairs (0,8)
 * and (4,12) that Sec. III-D uses for its early rejection. */
static const int kRingDx[16] = {0, 1, 2, 3, 3, 3, 2, 1, 0, -1, -2, -3, -3, -3, -2, -1};
static const int kRingDy[16] = {-3, -3, -2, -1, 0, 1, 2, 3, 3, 3, 2, 1, 0, -1, -2, -3};

extern "C" void vo_fast_ring(int32_t* dx, int32_t* dy) {
  for (int k = 0; k < 16; ++k) {
    dx[k] = kRingDx[k];
    dy[k] = kRingDy[k];
  }
}

/* Sec. III-D: FAST-9. A pixel p is a corner at tau if some 9 contiguous ring
 * pixels are all > I(p)+tau, or all < I(p)-tau; its score is the largest such
 * tau. With d_k = I_k - I(p), "all of arc A > I(p)+tau" is min_{k in A} d_k >
 * tau, so the largest qualifying integer tau for a bright arc is
 * min_{k in A} d_k - 1, and the score is the largest of these over the 16
 * arcs of length 9 and both polarities. Arcs longer than 9 contain an arc of
 * 9, so length-9 arcs suffice. tau is restricted to tau >= 0; a pixel with no
 * qualifying tau >= 0 scores -1 (not a corner). */
static int fast_score_at(const uint8_t* img, int pitch, int x, int y) {
  const int c = px(img, pitch, x, y);
  int d[16];
  for (int k = 0; k < 16; ++k) d[k] = px(img, pitch, x + kRingDx[k], y + kRingDy[k]) - c;
  int best = -1000;
  for (int start = 0; start < 16; ++start) {
    int min_bright = 1000, min_dark = 1000;
    for (int a = 0; a < 9; ++a) {
      const int dk = d[(start + a) % 16];
      min_bright = std::min(min_bright, dk);
      min_dark = std::min(min_dark, -dk);
    }
    best = std::max(best, std::max(min_bright, min_dark));
  }
  const int tau = best - 1;
  return tau >= 0 ? tau : -1;
}

extern "C" void vo_fast_scores(const uint8_t* img, int32_t w, int32_t h, int32_t pitch,
                               int16_t* score) {
  for (int y = 0; y < h; ++y) {
    for (int x = 0; x < w; ++x) {
      const bool inside = x >= 3 && x <= w - 4 && y >= 3 && y <= h - 4;
      score[(long)y * w + x] = (int16_t)(inside ? fast_score_at(img, pitch, x, y) : -1);
    }
  }
}

namespace {
struct Cand {
  int score, x, y;
};
/* Per-cell order: score descending, then y ascending, then x ascending (the
 * paper's sort leaves ties open; this fixes one order). */
bool cand_before(const Cand& a, const Cand& b) {
  if (a.score != b.score) return a.score > b.score;
  if (a.y != b.y) return a.y < b.y;
  return a.x < b.x;
}
}  // namespace

/* Sec. III-D: per cell, for each threshold T of the sequence in turn: take
 * the corners with score >= T, keep the strict 3x3 local maxima (NMS), and
 * if at least k remain keep the strongest k and stop; otherwise continue
 * with the next threshold, and after the last one keep all that remain.
 * k is reduced by the cell's count of existing tracks (the mask/cell buffers
 * of Sec. III-B). NMS compares against the 8 image neighbours, in this cell
 * or the next, with non-corners scoring -1; an equal neighbour suppresses.
 * Cells: the full cells of a grid anchored at (0,0).
 *
 * one_pass = 1 computes the same result the short way: the top k of all
 * local maxima with score >= the last threshold (the sets S_T are nested and
 * NMS does not depend on T). The tests check that both agree. */
extern "C" int32_t vo_detect_grid(const uint8_t* img, int32_t w, int32_t h, int32_t pitch,
                                  const vo_detect_params* p, const uint8_t* occupancy,
                                  const uint8_t* mask, int32_t mask_pitch, float* kp_xy,
                                  int16_t* kp_score, int32_t capacity, int32_t one_pass) {
  std::vector<int16_t> score((size_t)w * h);
  vo_fast_scores(img, w, h, pitch, score.data());
  auto sc = [&](int x, int y) -> int {
    if (x < 0 || y < 0 || x >= w || y >= h) return -1;
    return score[(size_t)y * w + x];
  };
  auto is_local_max = [&](int x, int y) -> bool {
    const int s = sc(x, y);
    if (s < 0) return false;
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx)
        if ((dx || dy) && sc(x + dx, y + dy) >= s) return false;
    return true;
  };
  const int gx = w / p->cell_w, gy = h / p->cell_h;
  int n_out = 0;
  for (int cy = 0; cy < gy; ++cy) {
    for (int cx = 0; cx < gx; ++cx) {
      const int occ = occupancy ? occupancy[cy * gx + cx] : 0;
      const int k_eff = p->k - occ;
      if (k_eff <= 0) continue;
      std::vector<Cand> chosen;
      const int t_first = one_pass ? p->n_thresholds - 1 : 0;
      for (int ti = t_first; ti < p->n_thresholds; ++ti) {
        const int T = p->thresholds[ti];
        std::vector<Cand> st;
        for (int y = cy * p->cell_h; y < (cy + 1) * p->cell_h; ++y) {
          for (int x = cx * p->cell_w; x < (cx + 1) * p->cell_w; ++x) {
            if (x < p->border || x > w - 1 - p->border || y < p->border || y > h - 1 - p->border)
              continue;
            if (mask && mask[(long)y * mask_pitch + x] == 0) continue;
            if (sc(x, y) < T) continue;
            if (!is_local_max(x, y)) continue;
            st.push_back({sc(x, y), x, y});
          }
        }
        std::sort(st.begin(), st.end(), cand_before);
        if ((int)st.size() >= k_eff) {
          chosen.assign(st.begin(), st.begin() + k_eff);
          break;
        }
        if (ti == p->n_thresholds - 1) chosen = st;
      }
      for (const Cand& c : chosen) {
        if (n_out >= capacity) return n_out;
        kp_xy[2 * n_out] = (float)c.x;
        kp_xy[2 * n_out + 1] = (float)c.y;
        kp_score[n_out] = (int16_t)c.score;
        ++n_out;
      }
    }
  }
  return n_out;
}
