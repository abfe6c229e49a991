// Learned flow initializer: inference and training kernels (device code of
// the network in initnet_dev.cuh).
//
//  pack     FP32 master parameters -> BF16 [N][K] matrices + FP32 biases
//  extract  network inputs of keypoints from two pyramids
//  forward  persistent CTAs of 128 threads over rounds of 32 samples, layer
//           by layer on the tcgen05 tensor cores (initnet_tc.cuh: BF16
//           operands in shared memory, FP32 accumulators in tensor memory)
//  train    the forward pass of one sample per warp (same layers, BF16
//           activations), then the backward pass in FP32 per warp, with
//           the weight gradients summed in shared memory per CTA and added to
//           the global gradient once per CTA
//  adam     Adam update of the master parameters
#include <math.h>

#include "initnet_dev.cuh"
#include "initnet_tc.cuh"
#include "initnet_train_dev.cuh"

namespace vio {
namespace {

using namespace net;

__global__ void pack_kernel(const float* __restrict__ m, uint16_t* __restrict__ w,
                            float* __restrict__ b) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < N_BF16) {
    float v = 0.f;
    if (i < OFF_W2) {                     // w1: [32][48], taps 36..47 zero
      const int n = i / K1, k = i % K1;
      if (k < 36) v = m[M_W1 + n * 36 + k];
    } else if (i < OFF_W3) {
      v = m[M_W2 + (i - OFF_W2)];
    } else if (i < OFF_W4) {
      v = m[M_W3 + (i - OFF_W3)];
    } else if (i < OFF_W5) {
      v = m[M_W4 + (i - OFF_W4)];
    } else {                              // w5: [8][64], rows 3..7 zero
      const int n = (i - OFF_W5) / K5, k = (i - OFF_W5) % K5;
      if (n < 3) v = m[M_W5 + n * K5 + k];
    }
    w[i] = f2bf(v);
  }
  if (i < N_BIAS) {
    float v = 0.f;
    if (i < OFF_B2) v = m[M_B1 + i];
    else if (i < OFF_B3) v = m[M_B2 + i - OFF_B2];
    else if (i < OFF_B4) v = m[M_B3 + i - OFF_B3];
    else if (i < OFF_B5) v = m[M_B4 + i - OFF_B4];
    else if (i < OFF_B5 + 3) v = m[M_B5 + i - OFF_B5];
    b[i] = v;
  }
}

struct ExtractArgs {
  Geom g;
  Batch src, dst;
  const float* pts;
  const int32_t* count;
  int capacity, la, lb;
  uint16_t* x;   // [n][4][16][16] bf16
};

__global__ void extract_kernel(ExtractArgs a) {
  __shared__ __align__(16) uint8_t smem[4][WARP_SMEM];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long wid = (long long)blockIdx.x * 4 + warp;
  const long long total = (long long)a.capacity * a.src.n;
  if (wid >= total) return;
  const int img = (int)(wid / a.capacity);
  const int k = (int)(wid - (long long)img * a.capacity);
  const int n = a.count ? min(a.count[img], a.capacity) : a.capacity;
  uint16_t* out = a.x + wid * 1024;
  if (k >= n) {
    for (int e = lane; e < 1024; e += 32) out[e] = 0;
    return;
  }
  uint8_t* ws = smem[warp];
  extract_warp(a.g, a.src, img, a.dst, img, a.pts[2 * wid], a.pts[2 * wid + 1], a.la, a.lb, ws,
               lane);
  const uint16_t* xb = reinterpret_cast<const uint16_t*>(ws + S_X);
  for (int e = lane; e < 1024; e += 32) {
    const int ch = e >> 8, r = (e >> 4) & 15, c = e & 15;
    out[e] = xb[ch * XP * XP + (r + 1) * XP + (c + 1)];
  }
}

// Status word of the tensor-core forward passes (VIO_ERR_TIMEOUT when one
// gave up waiting for an MMA completion).
__device__ int32_t g_net_fault;

// Inference over n inputs ([n][4][16][16] BF16): persistent CTAs over rounds
// of 32 samples.
__global__ void __launch_bounds__(ntc::THREADS, 1) forward_tc_kernel(
    const void* __restrict__ packed_w, const uint16_t* __restrict__ x, int n,
    float* __restrict__ out, int32_t* fault) {
  extern __shared__ __align__(16) uint8_t sm[];
  const ntc::XSource src{x, n, out};
  ntc::run(src, packed_w, sm, fault);
}

__global__ void __launch_bounds__(TRAIN_WARPS * 32) train_kernel(
    const void* __restrict__ packed_w, const uint16_t* __restrict__ x,
    const float* __restrict__ flow, const int32_t* __restrict__ index, int n, float grad_scale,
    float radius, float* __restrict__ grad, float* __restrict__ loss_sum) {
  extern __shared__ __align__(16) uint8_t dsm[];
  train_block(packed_w, x, flow, index, n, grad_scale, radius, grad, loss_sum, dsm);
}

__global__ void adam_kernel(float* __restrict__ w, const float* __restrict__ g,
                            float* __restrict__ m, float* __restrict__ v, int n, float lr,
                            float b1, float b2, float eps, float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

}  // namespace

int32_t* net_fault_word() {
  static int32_t* addr[64] = {};
  static PerDeviceOnce once;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  once_per_device(once, [&] {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_net_fault);
    addr[dev] = static_cast<int32_t*>(p);
    return e;
  });
  return addr[dev];
}

int initnet_train_smem() { return net::train_smem_bytes(); }

}  // namespace vio

extern "C" vio_status vio_initnet_pack(const float* d_master, void* d_packed, void* stream) {
  using namespace vio::net;
  if (!d_master || !d_packed) return VIO_ERR_INVALID_ARG;
  uint8_t* p = reinterpret_cast<uint8_t*>(d_packed);
  vio::pack_kernel<<<(N_BF16 + 255) / 256, 256, 0, (cudaStream_t)stream>>>(
      d_master, reinterpret_cast<uint16_t*>(p), reinterpret_cast<float*>(p + OFF_B));
  return cudaGetLastError() == cudaSuccess ? VIO_OK : VIO_ERR_CUDA;
}

extern "C" vio_status vio_initnet_extract(const vio_pyr_layout* layout, const vio_pyr_batch* src,
                                          const vio_pyr_batch* dst, const float* d_pts,
                                          const int32_t* d_count, int32_t capacity,
                                          int32_t level_a, int32_t level_b, uint16_t* d_x,
                                          void* stream) {
  if (!layout || !src || !dst || !d_pts || !d_x || capacity < 0 ||
      src->n_images != dst->n_images || src->n_images < 1)
    return VIO_ERR_INVALID_ARG;
  if (level_a < 0 || level_b < 0 || level_a >= layout->n_levels || level_b >= layout->n_levels)
    return VIO_ERR_INVALID_ARG;
  if ((layout->n_levels > 1) && (!src->d_upper || !dst->d_upper)) return VIO_ERR_INVALID_ARG;
  vio::ExtractArgs a{vio::make_geom(*layout), vio::make_batch(*src), vio::make_batch(*dst),
                     d_pts, d_count, capacity, level_a, level_b, d_x};
  const long long warps = (long long)capacity * src->n_images;
  if (warps == 0) return VIO_OK;
  vio::extract_kernel<<<(unsigned)((warps + 3) / 4), 128, 0, (cudaStream_t)stream>>>(a);
  return cudaGetLastError() == cudaSuccess ? VIO_OK : VIO_ERR_CUDA;
}

extern "C" vio_status vio_initnet_forward(const void* d_packed, const uint16_t* d_x, int32_t n,
                                          float* d_out, void* stream) {
  using namespace vio::net;
  if (!d_packed || !d_x || !d_out || n < 0 || ((uintptr_t)d_packed & 15) ||
      ((uintptr_t)d_x & 15))
    return VIO_ERR_INVALID_ARG;
  if (n == 0) return VIO_OK;
  static vio::PerDeviceOnce attr;
  if (vio::once_per_device(attr, [] {
        return cudaFuncSetAttribute(vio::forward_tc_kernel,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, vio::ntc::SMEM);
      }) != cudaSuccess)
    return VIO_ERR_CUDA;
  const int rounds = (n + vio::ntc::ROUND - 1) / vio::ntc::ROUND, sms = vio::sm_count();
  vio::forward_tc_kernel<<<rounds < sms ? rounds : sms, vio::ntc::THREADS, vio::ntc::SMEM,
                           (cudaStream_t)stream>>>(d_packed, d_x, n, d_out,
                                                   vio::net_fault_word());
  return cudaGetLastError() == cudaSuccess ? VIO_OK : VIO_ERR_CUDA;
}

extern "C" vio_status vio_initnet_fault(int32_t* status) {
  if (!status) return VIO_ERR_INVALID_ARG;
  int32_t* w = vio::net_fault_word();
  if (!w) return VIO_ERR_CUDA;
  int32_t v = 0;
  if (cudaMemcpy(&v, w, sizeof(v), cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemset(w, 0, sizeof(v)) != cudaSuccess)
    return VIO_ERR_CUDA;
  *status = v;
  return VIO_OK;
}

extern "C" vio_status vio_initnet_train_step(const void* d_packed, const uint16_t* d_x,
                                             const float* d_flow, const int32_t* d_index,
                                             int32_t n, float grad_scale, float label_radius,
                                             float* d_grad, float* d_loss, void* stream) {
  if (!d_packed || !d_x || !d_flow || !d_grad || !d_loss || n < 0 || !(label_radius > 0.f))
    return VIO_ERR_INVALID_ARG;
  if (n == 0) return VIO_OK;
  const int smem = vio::initnet_train_smem();
  cudaError_t e = cudaFuncSetAttribute(vio::train_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return VIO_ERR_CUDA;
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int blocks = (int)std::min<long long>((long long)sms, (n + vio::TRAIN_WARPS - 1) /
                                                                  vio::TRAIN_WARPS);
  vio::train_kernel<<<blocks, vio::TRAIN_WARPS * 32, smem, (cudaStream_t)stream>>>(
      d_packed, d_x, d_flow, d_index, n, grad_scale, label_radius, d_grad, d_loss);
  return cudaGetLastError() == cudaSuccess ? VIO_OK : VIO_ERR_CUDA;
}

extern "C" vio_status vio_initnet_adam(float* d_master, const float* d_grad, float* d_m,
                                       float* d_v, int32_t step, float lr, float beta1,
                                       float beta2, float eps, void* stream) {
  if (!d_master || !d_grad || !d_m || !d_v || step < 1) return VIO_ERR_INVALID_ARG;
  const float c1 = 1.f - powf(beta1, (float)step), c2 = 1.f - powf(beta2, (float)step);
  const int n = vio::net::N_MASTER;
  vio::adam_kernel<<<(n + 255) / 256, 256, 0, (cudaStream_t)stream>>>(
      d_master, d_grad, d_m, d_v, n, lr, beta1, beta2, eps, c1, c2);
  return cudaGetLastError() == cudaSuccess ? VIO_OK : VIO_ERR_CUDA;
}

static_assert(VIO_INITNET_N_PARAMS == vio::net::N_MASTER, "master parameter count");
static_assert(VIO_INITNET_PACKED_BYTES == vio::net::PACKED_BYTES, "packed size");
