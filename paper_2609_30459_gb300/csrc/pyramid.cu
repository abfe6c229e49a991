// Image pyramid (Sec. III-C, Eq. 1-3): L_{l+1}(x,y) =
// round((sum_j w_j sum_i w_i L_l(2x+i, 2y+j)) / 256), w = [1,4,6,4,1],
// computed separably (Eq. 2 then Eq. 3) in integer arithmetic, edges clamped.
//
// One CTA of 256 threads makes a 64 x 16 tile of level l+1 from a
// 131 x 35 region of level l staged in shared memory; the horizontal pass
// (Eq. 2) goes to a second shared buffer, the vertical pass (Eq. 3) to
// global memory. All images of a batch and all tiles of a level are one
// launch; levels follow each other in stream order.
#include "common.cuh"

namespace vio {
namespace {

constexpr int TW = 64, TH = 16;            // output tile
constexpr int SW = 2 * TW + 3;             // source region width  (131)
constexpr int SH = 2 * TH + 3;             // source region height (35)
constexpr int THREADS = 256;

__global__ void __launch_bounds__(THREADS) pyr_down_kernel(Geom g, Batch b, int l,
                                                           int round_mode) {
  __shared__ uint8_t src_s[SH][SW + 1];
  __shared__ uint16_t hsum[SH][TW];        // Eq. 2: V = sum_i w_i L(2x+i, y) <= 4080

  const int img = blockIdx.z;
  const uint8_t* src = level_ptr(g, b, img, l);
  uint8_t* dst = level_ptr_mut(g, b, img, l + 1);
  const int W = g.w[l], H = g.h[l], P = g.pitch[l];
  const int w2 = g.w[l + 1], h2 = g.h[l + 1], P2 = g.pitch[l + 1];
  const int ox0 = blockIdx.x * TW, oy0 = blockIdx.y * TH;
  const int sx0 = 2 * ox0 - 2, sy0 = 2 * oy0 - 2;

  // stage the clamped source region
  for (int i = threadIdx.x; i < SH * SW; i += THREADS) {
    const int r = i / SW, c = i - r * SW;
    const int sy = min(max(sy0 + r, 0), H - 1);
    const int sx = min(max(sx0 + c, 0), W - 1);
    src_s[r][c] = src[(long long)sy * P + sx];
  }
  __syncthreads();

  // Eq. 2: horizontal pass at the even columns 2x of the tile
  for (int i = threadIdx.x; i < SH * TW; i += THREADS) {
    const int r = i / TW, x = i - r * TW;
    const uint8_t* s = &src_s[r][2 * x];
    hsum[r][x] = (uint16_t)(s[0] + 4 * s[1] + 6 * s[2] + 4 * s[3] + s[4]);
  }
  __syncthreads();

  // Eq. 3: vertical pass at the even rows 2y, then the rounding shift
  const int add = round_mode == 0 ? 128 : 0;
  for (int i = threadIdx.x; i < TH * TW; i += THREADS) {
    const int y = i / TW, x = i - y * TW;
    const int ox = ox0 + x, oy = oy0 + y;
    if (ox < w2 && oy < h2) {
      const uint32_t s = hsum[2 * y][x] + 4u * hsum[2 * y + 1][x] + 6u * hsum[2 * y + 2][x] +
                         4u * hsum[2 * y + 3][x] + hsum[2 * y + 4][x];
      dst[(long long)oy * P2 + ox] = (uint8_t)((s + add) >> 8);
    }
  }
}

}  // namespace

cudaError_t launch_pyramid(const Geom& g, const Batch& b, int round_mode, cudaStream_t s) {
  for (int l = 0; l + 1 < g.n_levels; ++l) {
    dim3 grid((g.w[l + 1] + TW - 1) / TW, (g.h[l + 1] + TH - 1) / TH, b.n);
    pyr_down_kernel<<<grid, THREADS, 0, s>>>(g, b, l, round_mode);
  }
  return cudaGetLastError();
}

}  // namespace vio
