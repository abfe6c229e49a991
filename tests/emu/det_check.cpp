// Grid-cell detection device code (detect_dev.cuh) run on the host, block by
// block, against the oracle's one-pass detection (test infrastructure).
// Every CTA's shared memory is a heap buffer of exactly the computed size, so
// AddressSanitizer reports any out-of-bounds shared or global access.
#include "blockemu.h"
#include "detect_dev.cuh"
#include "oracle.h"
#include <random>
using namespace vio;
using namespace vio::det;

struct Case { int w, h, cw, ch, k, nt, g, tmin, border; bool masked; int kind; int sel; };

static int run_case(const Case& C, std::mt19937& rng) {
  const int W = C.w, H = C.h, P = W + 16;
  std::vector<uint8_t> img((size_t)P * H);
  std::vector<float> f((size_t)W * H);
  for (auto& v : f) v = (float)(rng() % 256);
  for (int it = 0; it < 2; ++it) {          // two 3x3 box blurs: corner-rich texture
    std::vector<float> g2 = f;
    for (int y = 0; y < H; ++y)
      for (int x = 0; x < W; ++x) {
        float s = 0;
        int n = 0;
        for (int dy = -1; dy <= 1; ++dy)
          for (int dx = -1; dx <= 1; ++dx) {
            const int xx = x + dx, yy = y + dy;
            if (xx >= 0 && yy >= 0 && xx < W && yy < H) { s += f[yy * W + xx]; ++n; }
          }
        g2[y * W + x] = s / n;
      }
    f = g2;
  }
  for (int y = 0; y < H; ++y)
    for (int x = 0; x < W; ++x) {
      float v = (f[y * W + x] - 128) * 3 + 128;
      if (C.kind == 1) v = 120 + (f[y * W + x] - 128) * 0.25f;      // low contrast
      if (C.kind == 2) v = (float)(rng() % 256);                     // raw noise
      img[(size_t)y * P + x] = (uint8_t)std::min(255.f, std::max(0.f, v));
    }
  std::vector<uint8_t> mask((size_t)W * H, 1);
  if (C.masked) for (auto& v : mask) v = (rng() % 5) != 0;
  const int gx = W / C.cw, gy = H / C.ch, n_cells = gx * gy;
  CellGeom cg{C.cw, C.ch, gx, C.k, C.tmin, C.border, 1, 1, 1, C.sel};
  const int smem = detect_setup(cg, C.nt, C.g);
  if (smem < 0) return 1;
  std::vector<unsigned long long> cand((size_t)n_cells * C.k, 0);
  std::vector<int32_t> count(n_cells, -7);
  const int nblk = detect_blocks(gx, gy, cg.bcx, cg.bcy);
  for (int blk = 0; blk < nblk; ++blk) {
    uint8_t* sm = (uint8_t*)aligned_alloc(16, (smem + 15) & ~15);
    memset(sm, 0xa5, (smem + 15) & ~15);
    emu_run_block(C.nt, [&] {
      if (C.masked)
        detect_block<true>(img.data(), W, H, P, cg, gy, blk, mask.data(), cand.data(),
                           count.data(), sm);
      else
        detect_block<false>(img.data(), W, H, P, cg, gy, blk, nullptr, cand.data(),
                            count.data(), sm);
    }, EmuDim{(unsigned)blk, 0, 0});
    free(sm);
  }
  vo_detect_params dp{};
  dp.cell_w = C.cw; dp.cell_h = C.ch; dp.k = C.k; dp.n_thresholds = 1;
  dp.thresholds[0] = C.tmin; dp.border = C.border;
  const int cap = n_cells * C.k;
  std::vector<float> kp(2 * (size_t)cap + 2);
  std::vector<int16_t> sc(cap + 1);
  const int n = vo_detect_grid(img.data(), W, H, P, &dp, nullptr, C.masked ? mask.data() : nullptr,
                               W, kp.data(), sc.data(), cap, 1);
  std::vector<std::vector<unsigned long long>> ref(n_cells);
  for (int i = 0; i < n; ++i) {
    const int x = (int)kp[2 * i], y = (int)kp[2 * i + 1];
    ref[(y / C.ch) * gx + x / C.cw].push_back(((unsigned long long)sc[i] << 32) |
                                               (unsigned)(~(unsigned)(y * W + x)));
  }
  int bad = 0;
  for (int c = 0; c < n_cells; ++c) {
    bool same = count[c] == (int)ref[c].size();
    for (int j = 0; same && j < count[c]; ++j) same = cand[(size_t)c * C.k + j] == ref[c][j];
    bad += !same;
  }
  printf("%dx%d cells %dx%d k%d nt%d g%d sel%d T%d: %d keypoints, %d cells differ\n", W, H, C.cw,
         C.ch, C.k, C.nt, cg.g, C.sel, C.tmin, n, bad);
  return bad;
}

int main(int argc, char** argv) {
  std::mt19937 rng(argc > 1 ? atoi(argv[1]) : 5);
  const std::vector<Case> cases = {
      {160, 120, 37, 32, 1, 128, 1, 5, 9, false, 0, 0},
      {160, 120, 40, 30, 2, 256, 8, 5, 0, true, 0, 1},
      {120, 96, 40, 32, 1, 128, 4, 0, 3, false, 0, 2},
      {128, 96, 64, 48, 3, 256, 2, 5, 0, true, 2, 0},   // raw noise: queues overflow
      {97, 61, 7, 5, 2, 256, 8, 10, 2, false, 1, 0},
      {64, 9, 2, 3, 1, 128, 2, 5, 1, true, 2, 1},
  };
  int fails = 0;
  for (const auto& c : cases) fails += run_case(c, rng);
  printf("FAILS %d\n", fails);
  return fails != 0;
}
