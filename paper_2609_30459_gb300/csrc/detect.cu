// Grid-cell FAST-9 detection entry points (Sec. III-D): the per-pixel score
// map, the per-cell candidate kernel (one to eight warps per cell, chosen
// from the launch size, blocks of cells per CTA; device code in
// detect_dev.cuh) and the
// per-image selection that applies k_eff = k - occupancy and writes the
// survivors in cell raster order with a block-wide prefix sum.
#include "detect_dev.cuh"

namespace vio {
namespace {

__global__ void fast_scores_kernel(const uint8_t* __restrict__ img, int w, int h, int pitch,
                                   int16_t* __restrict__ out) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= w || y >= h) return;
  int s = -1;
  if (x >= 3 && x <= w - 4 && y >= 3 && y <= h - 4) {
    int v[16];
#pragma unroll
    for (int k = 0; k < 16; ++k)
      v[k] = __ldg(img + (long long)(y + det::ring_dy(k)) * pitch + x + det::ring_dx(k));
    s = det::fast_m(v, __ldg(img + (long long)y * pitch + x)) - 1;
  }
  out[(long long)y * w + x] = (int16_t)s;
}

struct DetectArgs {
  Geom g;
  Batch b;
  const uint8_t* mask;
  long long mask_stride;
  unsigned long long* cand;   // [img][cell][k]
  int32_t* cand_count;        // [img][cell]
  det::CellGeom cg;
  int n_cells, gy;
};

__global__ void __launch_bounds__(det::kThreads, 6) detect_cells_kernel(DetectArgs a) {
  extern __shared__ __align__(16) uint8_t smem[];
  const int img = blockIdx.y;
  const uint8_t* src = level_ptr(a.g, a.b, img, 0);
  unsigned long long* cand = a.cand + (long long)img * a.n_cells * a.cg.k;
  int32_t* count = a.cand_count + (long long)img * a.n_cells;
  if (a.mask)
    det::detect_block<true>(src, a.g.w[0], a.g.h[0], a.g.pitch[0], a.cg, a.gy, blockIdx.x,
                            a.mask + (long long)img * a.mask_stride, cand, count, smem);
  else
    det::detect_block<false>(src, a.g.w[0], a.g.h[0], a.g.pitch[0], a.cg, a.gy, blockIdx.x,
                             nullptr, cand, count, smem);
}

constexpr int SEL_THREADS = 512;

__global__ void __launch_bounds__(SEL_THREADS) select_kernel(
    const unsigned long long* __restrict__ cand, const int32_t* __restrict__ cand_count,
    const uint8_t* __restrict__ occ, int n_cells, int k, int W, float* __restrict__ kp,
    int16_t* __restrict__ score, int32_t* __restrict__ count, int capacity) {
  __shared__ int warp_sums[SEL_THREADS / 32];
  __shared__ int carry_s;
  const int img = blockIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned long long* ci = cand + (long long)img * n_cells * k;
  const int32_t* cc = cand_count + (long long)img * n_cells;
  const uint8_t* oc = occ ? occ + (long long)img * n_cells : nullptr;
  float* kpo = kp + (long long)img * capacity * 2;
  int16_t* so = score + (long long)img * capacity;
  if (threadIdx.x == 0) carry_s = 0;
  __syncthreads();
  for (int base = 0; base < n_cells; base += SEL_THREADS) {
    const int cell = base + threadIdx.x;
    int nsel = 0;
    if (cell < n_cells) {
      const int keff = k - (oc ? (int)oc[cell] : 0);
      nsel = max(0, min(keff, (int)cc[cell]));
    }
    // block exclusive scan of nsel
    int incl = nsel;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    if (lane == 31) warp_sums[warp] = incl;
    __syncthreads();
    if (warp == 0) {
      int ws = lane < SEL_THREADS / 32 ? warp_sums[lane] : 0;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, ws, o);
        if (lane >= o) ws += t;
      }
      if (lane < SEL_THREADS / 32) warp_sums[lane] = ws;   // inclusive per warp
    }
    __syncthreads();
    const int carry = carry_s;
    const int excl = carry + (warp ? warp_sums[warp - 1] : 0) + incl - nsel;
    for (int r = 0; r < nsel; ++r) {
      const int o = excl + r;
      if (o < capacity) {
        const unsigned long long key = ci[(long long)cell * k + r];
        const unsigned idx = ~(unsigned)(key & 0xffffffffu);
        kpo[2 * o] = (float)(idx % (unsigned)W);
        kpo[2 * o + 1] = (float)(idx / (unsigned)W);
        so[o] = (int16_t)(key >> 32);
      }
    }
    __syncthreads();
    if (threadIdx.x == SEL_THREADS - 1) carry_s = carry + warp_sums[SEL_THREADS / 32 - 1];
    __syncthreads();
  }
  if (threadIdx.x == 0) count[img] = min(carry_s, capacity);
}

}  // namespace

cudaError_t launch_fast_scores(const uint8_t* img, int w, int h, int pitch, int16_t* out,
                               cudaStream_t s) {
  dim3 blk(32, 8);
  dim3 grid((w + 31) / 32, (h + 7) / 8);
  fast_scores_kernel<<<grid, blk, 0, s>>>(img, w, h, pitch, out);
  return cudaGetLastError();
}

cudaError_t launch_detect(const vio_params& p, const Geom& g, const Batch& b,
                          const uint8_t* occ, const uint8_t* mask, long long mask_stride,
                          unsigned long long* cand, int32_t* cand_count, float* kp,
                          int16_t* score, int32_t* count, int capacity, cudaStream_t s) {
  DetectArgs a;
  a.g = g;
  a.b = b;
  a.mask = mask;
  a.mask_stride = mask_stride;
  a.cand = cand;
  a.cand_count = cand_count;
  a.cg = det::CellGeom{p.cell_w, p.cell_h, g.w[0] / p.cell_w, p.k_per_cell,
                       p.thresholds[p.n_thresholds - 1], p.detect_border, 1, 1, 1,
                       p.select_mode};
  a.gy = g.h[0] / p.cell_h;
  const int n_cells = a.cg.gx * a.gy;
  a.n_cells = n_cells;
  const int smem = det::detect_setup(
      a.cg, det::kThreads, det::warps_per_cell((long long)n_cells * b.n, sm_count()));
  if (smem < 0) return cudaErrorInvalidValue;
  if (n_cells > 0) {
    // as much shared memory as the SM has: more CTAs (once per device)
    static PerDeviceOnce carveout;
    const cudaError_t ec = once_per_device(carveout, [] {
      return cudaFuncSetAttribute(detect_cells_kernel,
                                  cudaFuncAttributePreferredSharedMemoryCarveout,
                                  (int)cudaSharedmemCarveoutMaxShared);
    });
    if (ec != cudaSuccess) return ec;
    if (smem > 48 * 1024) {
      cudaError_t e = cudaFuncSetAttribute(detect_cells_kernel,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
      if (e != cudaSuccess) return e;
    }
    dim3 grid(det::detect_blocks(a.cg.gx, a.gy, a.cg.bcx, a.cg.bcy), b.n);
    detect_cells_kernel<<<grid, det::kThreads, smem, s>>>(a);
  }
  return launch_select(cand, cand_count, occ, n_cells, a.cg.k, g.w[0], kp, score, count,
                       capacity, b.n, s);
}

cudaError_t launch_select(const unsigned long long* cand, const int32_t* cand_count,
                          const uint8_t* occ, int n_cells, int k, int w, float* kp,
                          int16_t* score, int32_t* count, int capacity, int n_images,
                          cudaStream_t s) {
  select_kernel<<<n_images, SEL_THREADS, 0, s>>>(cand, cand_count, occ, n_cells, k, w, kp, score,
                                                 count, capacity);
  return cudaGetLastError();
}

}  // namespace vio
