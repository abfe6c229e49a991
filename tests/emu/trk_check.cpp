// The patch tracker's device code (track_dev.cuh: templates, Gauss-Newton
// steps, the forward-backward check) run on the host with emulated warps
// (test infrastructure), so that its reads are checked by AddressSanitizer
// and its results can be compared with the FP64 oracle without a GPU. The two
// images' levels sit in one batch as on the device, each level between
// poisoned gaps, so that a read outside any level is reported. argv[1] holds
//   int32 n_levels, n_points, gn_iters; float32 fb_max_dist;
//   per level: int32 w, h, then w*h source bytes and w*h target bytes;
//   n_points x float32 (x, y, init_x, init_y, has_init);
// argv[2] receives n_points x float32 (status, x, y, theta, fb_dist), with
// NaN position and angle where the forward pass gave no result.
#include "blockemu.h"
#include "track_dev.cuh"

#include <sanitizer/asan_interface.h>

#include <vector>

using namespace vio;

namespace {
constexpr long long kGap = 64;   // poisoned bytes around every level
}

int main(int argc, char** argv) {
  if (argc < 3) return 2;
  FILE* f = fopen(argv[1], "rb");
  if (!f) return 2;
  int32_t hdr[3];
  float fb_max = 0.f;
  if (fread(hdr, 4, 3, f) != 3 || fread(&fb_max, 4, 1, f) != 1) return 2;
  const int L = hdr[0], n = hdr[1], iters = hdr[2];
  if (L < 1 || L > VIO_MAX_LEVELS || n < 0) return 2;
  Geom g{};
  g.n_levels = L;
  std::vector<std::vector<uint8_t>> px(2 * L);
  long long up_block = kGap;      // one image's upper levels, gaps between
  for (int l = 0; l < L; ++l) {
    int32_t wh[2];
    if (fread(wh, 4, 2, f) != 2) return 2;
    g.w[l] = wh[0];
    g.h[l] = wh[1];
    g.pitch[l] = wh[0];
    for (int img = 0; img < 2; ++img) {
      px[2 * l + img].resize((size_t)wh[0] * wh[1]);
      if (fread(px[2 * l + img].data(), 1, px[2 * l + img].size(), f) != px[2 * l + img].size())
        return 2;
    }
    if (l > 0) {
      g.off[l] = up_block;
      up_block += (long long)wh[0] * wh[1] + kGap;
    }
  }
  std::vector<float> pts((size_t)n * 5);
  if (fread(pts.data(), 4, pts.size(), f) != pts.size()) return 2;
  fclose(f);

  // level 0 of image i at l0 + i * l0_stride, level l >= 1 at
  // upper + i * upper_stride + off[l]; every byte between levels poisoned
  const long long s0 = (long long)g.w[0] * g.h[0];
  std::vector<uint8_t> l0buf((size_t)(kGap + 2 * (s0 + kGap)));
  std::vector<uint8_t> upbuf((size_t)(2 * up_block + kGap));
  Batch b{};
  b.l0 = l0buf.data() + kGap;
  b.l0_stride = s0 + kGap;
  b.upper = upbuf.data();
  b.upper_stride = up_block;
  b.n = 2;
  ASAN_POISON_MEMORY_REGION(l0buf.data(), l0buf.size());
  ASAN_POISON_MEMORY_REGION(upbuf.data(), upbuf.size());
  for (int img = 0; img < 2; ++img)
    for (int l = 0; l < L; ++l) {
      uint8_t* dst = l == 0 ? const_cast<uint8_t*>(b.l0) + img * b.l0_stride
                            : b.upper + img * b.upper_stride + g.off[l];
      ASAN_UNPOISON_MEMORY_REGION(dst, px[2 * l + img].size());
      memcpy(dst, px[2 * l + img].data(), px[2 * l + img].size());
    }

  std::vector<float> out((size_t)n * 5, 0.f);
  const TrackCfg cfg{iters, 1, fb_max, -1};
  gridDim.x = 1;
  for (int k = 0; k < n; ++k) {
    const float* q = &pts[(size_t)k * 5];
    float res[5];
    emu_run_block(32, [&] {
      const int lane = threadIdx.x & 31;
      trk::Pos tf{};
      float thf = 0.f, dist = 0.f, last = 0.f;
      bool have = false;
      const int st = trk::track_fb(g, b, 0, b, 1, q[0], q[1], q[4] != 0.f, q[2], q[3], 0.f, cfg,
                                   L - 1, lane, tf, thf, have, dist, last);
      if (lane == 0) {
        res[0] = (float)st;
        res[1] = have ? (float)tf.ax + tf.dx : std::nanf("");
        res[2] = have ? (float)tf.ay + tf.dy : std::nanf("");
        res[3] = have ? thf : std::nanf("");
        res[4] = dist;
      }
    }, EmuDim{0, 0, 0});
    for (int i = 0; i < 5; ++i) out[(size_t)k * 5 + i] = res[i];
  }
  f = fopen(argv[2], "wb");
  fwrite(out.data(), 4, out.size(), f);
  fclose(f);
  printf("points %d\n", n);
  return 0;
}
