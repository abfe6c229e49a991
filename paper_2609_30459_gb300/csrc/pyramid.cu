// Image pyramid entry point (Sec. III-C, Eq. 1-3). Levels are produced by
// passes of up to two levels each (device code in pyramid_dev.cuh): the
// first pass reads level 0 and writes levels 1-2, the next reads level 2 and
// writes levels 3-4, and so on; each pass is one launch over all tiles of all
// images.
#include "pyramid_dev.cuh"

namespace vio {
namespace {

__global__ void __launch_bounds__(pyr::kThreads) pyr_pass_kernel(Geom g, Batch b, int s, int m,
                                                                 int T, int ntx, int nty,
                                                                 int round_mode) {
  extern __shared__ __align__(16) uint8_t smem[];
  const int tiles = ntx * nty;
  const int img = blockIdx.x / tiles;
  const int t = blockIdx.x - img * tiles;
  const int ty = t / ntx, tx = t - ty * ntx;
  pyr::pyramid_pass(g, b, img, s, m, T, tx, ty, ntx, nty, round_mode, smem);
}

}  // namespace

cudaError_t launch_pyramid_from(const Geom& g, const Batch& b, int s0, int round_mode,
                                cudaStream_t st) {
  for (int s = s0; s + 1 < g.n_levels; s += pyr::kRestPass) {
    const int m = pyr::rest_pass_levels(g.n_levels, s);
    const int T = pyr::top_tile(m, pyr::kRestShift);
    int ntx, nty;
    pyr::pass_tiles(g.w, g.h, s, m, T, ntx, nty);
    const int smem = pyr::pass_smem_max(g.w, g.h, s, m, T);
    if (smem > 48 * 1024) {
      cudaError_t e = cudaFuncSetAttribute(pyr_pass_kernel,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
      if (e != cudaSuccess) return e;
    }
    const long long blocks = (long long)ntx * nty * b.n;
    pyr_pass_kernel<<<(unsigned)blocks, pyr::kThreads, smem, st>>>(g, b, s, m, T, ntx, nty,
                                                                   round_mode);
  }
  return cudaGetLastError();
}

cudaError_t launch_pyramid(const Geom& g, const Batch& b, int round_mode, cudaStream_t s) {
  return launch_pyramid_from(g, b, 0, round_mode, s);
}

}  // namespace vio
