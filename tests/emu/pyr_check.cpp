// Pyramid pass device code (pyramid_dev.cuh) run on the host, tile by tile,
// against the oracle's level-by-level filter (test infrastructure). Each
// tile's shared memory is a heap buffer of exactly its plan's size (and the
// launch's size must cover every tile's), so AddressSanitizer reports any
// out-of-bounds access.
#include "blockemu.h"
#include "pyramid_dev.cuh"
#include "oracle.h"
#include <random>
using namespace vio;

int main(int argc, char** argv) {
  std::mt19937 rng(argc > 1 ? atoi(argv[1]) : 1);
  const int NT = 32;
  const int sizes[][2] = {{160, 120}, {37, 29}, {17, 9}, {3, 5}, {100, 3}, {130, 66}};
  int fails = 0, cases = 0;
  for (const auto& sz : sizes)
    for (int L = 2; L <= 5; L += 3)
      for (int rm = 0; rm < 2; ++rm)
        for (int shift = -1; shift <= 1; shift += 2)
          for (int first = 1; first <= 4; first += 3) {
            const int w = sz[0], h = sz[1];
            int ws[8], hs[8];
            ws[0] = w;
            hs[0] = h;
            bool ok = true;
            for (int l = 1; l < L; ++l) {
              ws[l] = ws[l - 1] / 2;
              hs[l] = hs[l - 1] / 2;
              if (ws[l] < 1 || hs[l] < 1) ok = false;
            }
            if (!ok) continue;
            Geom g{};
            g.n_levels = L;
            const int pitch0 = w + (int)(rng() % 3) * 7;
            long long off = 0;
            for (int l = 0; l < L; ++l) { g.w[l] = ws[l]; g.h[l] = hs[l]; }
            g.pitch[0] = pitch0;
            for (int l = 1; l < L; ++l) {
              g.pitch[l] = (ws[l] + 127) & ~127;
              g.off[l] = off;
              off += ((long long)g.pitch[l] * hs[l] + 255) & ~255LL;
            }
            std::vector<uint8_t> l0((size_t)pitch0 * h);
            for (auto& v : l0) v = rng() & 0xff;
            std::vector<uint8_t> up(off > 0 ? off : 16, 0xcd);
            Batch b{l0.data(), 0, up.data(), 0, 1};
            // the launchers' passes: a first pass of `first` levels, then two each
            int s = 0;
            bool firstpass = true;
            while (s + 1 < L) {
              const int m = firstpass ? std::min(first, L - 1) : pyr::rest_pass_levels(L, s);
              const int T = pyr::top_tile(m, firstpass ? shift : pyr::kRestShift);
              int ntx, nty;
              pyr::pass_tiles(g.w, g.h, s, m, T, ntx, nty);
              const int smax = pyr::pass_smem_max(g.w, g.h, s, m, T);
              for (int ty = 0; ty < nty; ++ty)
                for (int tx = 0; tx < ntx; ++tx) {
                  const pyr::PassPlan P = pyr::pass_plan(g.w, g.h, s, m, T, tx, ty, ntx, nty);
                  if (P.total > smax) { printf("launch shared memory below a tile's\n"); return 1; }
                  uint8_t* smem = (uint8_t*)aligned_alloc(16, P.total + 16);
                  emu_run_block(NT, [&] { pyr::pyramid_pass(g, b, 0, s, m, T, tx, ty, ntx, nty, rm, smem); },
                                EmuDim{0, 0, 0});
                  free(smem);
                }
              s += m;
              firstpass = false;
            }
            // the oracle's levels, one from the other
            std::vector<uint8_t> cur((size_t)w * h);
            for (int y = 0; y < h; ++y) memcpy(&cur[(size_t)y * w], &l0[(size_t)y * pitch0], w);
            int cw = w, ch = h;
            ++cases;
            for (int l = 1; l < L; ++l) {
              std::vector<uint8_t> nxt((size_t)ws[l] * hs[l]);
              vo_pyr_down(cur.data(), cw, ch, cw, nxt.data(), ws[l], rm);
              bool same = true;
              for (int y = 0; y < hs[l] && same; ++y)
                same = memcmp(&up[g.off[l] + (size_t)y * g.pitch[l]], &nxt[(size_t)y * ws[l]], ws[l]) == 0;
              if (!same) {
                printf("%dx%d L%d round %d shift %d first %d: level %d differs\n", w, h, L, rm, shift,
                       first, l);
                ++fails;
                break;
              }
              cur = nxt;
              cw = ws[l];
              ch = hs[l];
            }
          }
  printf("cases %d FAILS %d\n", cases, fails);
  return fails != 0;
}
