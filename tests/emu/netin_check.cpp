// The flow network's input extraction on the host (test infrastructure):
// both device forms, run against pyramids whose levels sit between
// ASan-poisoned gaps with the device's alignment (upper levels 128-byte
// aligned, pitch a multiple of 128 bytes):
//  * net::extract_warp, one emulated warp per keypoint, BF16 into the
//    bordered input buffer;
//  * the prefetch path of the frame step's network launch: net::row_prefetch
//    (five aligned words per row), ntc::row_bytes (the row's 16 bytes, 0x80
//    outside the level) and ntc::byte_bf (a byte to (v - 128) / 64 in BF16).
// argv[1] holds int32 n_levels, n_points, la, lb; per level int32 w, h, then
// w*h source bytes and w*h target bytes; n_points x float32 (x, y). argv[2]
// receives, per point, the 4 x 16 x 16 BF16 values of each form in turn.
#include "blockemu.h"
#include "initnet_tc.cuh"

#include <sanitizer/asan_interface.h>

#include <vector>

using namespace vio;

namespace {
constexpr long long kGap = 128;   // poisoned bytes around every level
long long up128(long long v) { return (v + 127) & ~127LL; }
}  // namespace

int main(int argc, char** argv) {
  if (argc < 3) return 2;
  FILE* f = fopen(argv[1], "rb");
  if (!f) return 2;
  int32_t hdr[4];
  if (fread(hdr, 4, 4, f) != 4) return 2;
  const int L = hdr[0], n = hdr[1], la = hdr[2], lb = hdr[3];
  if (L < 2 || L > VIO_MAX_LEVELS || n < 0 || la < 1 || lb < 1 || la >= L || lb >= L) return 2;
  Geom g{};
  g.n_levels = L;
  std::vector<std::vector<uint8_t>> px(2 * L);
  long long up_block = kGap;
  for (int l = 0; l < L; ++l) {
    int32_t wh[2];
    if (fread(wh, 4, 2, f) != 2) return 2;
    g.w[l] = wh[0];
    g.h[l] = wh[1];
    g.pitch[l] = l == 0 ? wh[0] : (int)up128(wh[0]);
    for (int img = 0; img < 2; ++img) {
      px[2 * l + img].resize((size_t)wh[0] * wh[1]);
      if (fread(px[2 * l + img].data(), 1, px[2 * l + img].size(), f) != px[2 * l + img].size())
        return 2;
    }
    if (l > 0) {
      g.off[l] = up_block;
      up_block = up128(up_block + (long long)g.pitch[l] * wh[1]) + kGap;
    }
  }
  std::vector<float> pts((size_t)n * 2);
  if (fread(pts.data(), 4, pts.size(), f) != pts.size()) return 2;
  fclose(f);

  const long long s0 = (long long)g.w[0] * g.h[0];
  std::vector<uint8_t> l0buf((size_t)(kGap + 2 * (s0 + kGap)));
  // 128-byte aligned upper levels: over-allocate and align the base
  std::vector<uint8_t> upraw((size_t)(2 * up_block + kGap + 128));
  uint8_t* up = reinterpret_cast<uint8_t*>(up128((long long)(uintptr_t)upraw.data()));
  Batch b{};
  b.l0 = l0buf.data() + kGap;
  b.l0_stride = s0 + kGap;
  b.upper = up;
  b.upper_stride = up_block;
  b.n = 2;
  ASAN_POISON_MEMORY_REGION(l0buf.data(), l0buf.size());
  ASAN_POISON_MEMORY_REGION(upraw.data(), upraw.size());
  for (int img = 0; img < 2; ++img)
    for (int l = 0; l < L; ++l) {
      const int w = g.w[l], h = g.h[l], pitch = g.pitch[l];
      uint8_t* dst = l == 0 ? const_cast<uint8_t*>(b.l0) + img * b.l0_stride
                            : b.upper + img * b.upper_stride + g.off[l];
      // the whole pitch of every row is the level's (the prefetch reads
      // aligned words that may pass the last pixel, never the pitch)
      ASAN_UNPOISON_MEMORY_REGION(dst, (size_t)pitch * h);
      for (int y = 0; y < h; ++y) {
        memcpy(dst + (size_t)y * pitch, px[2 * l + img].data() + (size_t)y * w, w);
        memset(dst + (size_t)y * pitch + w, 0x5A, pitch - w);   // padding: must be ignored
      }
    }

  std::vector<uint16_t> out((size_t)n * 2 * 1024);
  std::vector<uint8_t> ws(net::WARP_SMEM);
  gridDim.x = 1;
  for (int k = 0; k < n; ++k) {
    const float x = pts[2 * k], y = pts[2 * k + 1];
    emu_run_block(32, [&] {
      const int lane = threadIdx.x & 31;
      net::clear_warp_smem(ws.data(), lane);
      net::extract_warp(g, b, 0, b, 1, x, y, la, lb, ws.data(), lane);
    }, EmuDim{0, 0, 0});
    const uint16_t* xb = reinterpret_cast<const uint16_t*>(ws.data() + net::S_X);
    uint16_t* o1 = &out[(size_t)k * 2048];
    uint16_t* o2 = o1 + 1024;
    for (int ch = 0; ch < 4; ++ch)
      for (int r = 0; r < 16; ++r)
        for (int c = 0; c < 16; ++c)
          o1[ch * 256 + r * 16 + c] = xb[ch * net::XP * net::XP + (r + 1) * net::XP + (c + 1)];
    emu_run_block(32, [&] {
      if (threadIdx.x != 0) return;
      for (int ch = 0; ch < 4; ++ch)
        for (int r = 0; r < 16; ++r) {
          net::RowWords R;
          net::row_prefetch(R, g, b, ch & 1, ch < 2 ? la : lb, x, y, r);
          uint32_t w4[4];
          ntc::row_bytes(R, w4);
          for (int c = 0; c < 16; ++c)
            o2[ch * 256 + r * 16 + c] =
                (uint16_t)(ntc::byte_bf(w4[c >> 2], (uint32_t)(c & 3)) >> 16);
        }
    }, EmuDim{0, 0, 0});
  }
  f = fopen(argv[2], "wb");
  fwrite(out.data(), 2, out.size(), f);
  fclose(f);
  printf("inputs %d\n", n);
  return 0;
}
